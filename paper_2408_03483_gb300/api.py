"""Python front end of the CUDA TT finite-volume library.

Device memory comes from PyTorch (cores, workspaces); the functions here only
marshal arguments to the C ABI (include/tt_fv.h) -- the names match it.
"""
import ctypes

import torch

from . import capi as C

C_ = C


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("paper_2408_03483_gb300 needs a CUDA device; there is no CPU path")


class DevTT:
    """A 2-D TT with device cores a (n1 x cap) and b (n2 x cap), column-major
    (stored as torch tensors of shape (cap, n1) / (cap, n2), row k = column k)."""

    def __init__(self, n1, n2, cap, device="cuda", rank=0):
        self.n1, self.n2, self.cap = int(n1), int(n2), int(cap)
        self.a = torch.zeros((self.cap, self.n1), dtype=torch.float64, device=device)
        self.b = torch.zeros((self.cap, self.n2), dtype=torch.float64, device=device)
        self.rank = int(rank)

    @classmethod
    def from_cores(cls, A, B, cap=None, device="cuda"):
        """From host/numpy cores A (n1 x r), B (n2 x r)."""
        A = torch.as_tensor(A, dtype=torch.float64)
        B = torch.as_tensor(B, dtype=torch.float64)
        r = A.shape[1]
        t = cls(A.shape[0], B.shape[0], cap or r, device=device, rank=r)
        t.a[:r].copy_(A.T.contiguous())
        t.b[:r].copy_(B.T.contiguous())
        return t

    def struct(self):
        return C.tt2(self.n1, self.n2, self.rank, self.cap, self.a.data_ptr(), self.b.data_ptr())

    def cores(self):
        """(A, B) as float64 CPU tensors of shape (n1, r), (n2, r)."""
        r = self.rank
        return self.a[:r].T.cpu(), self.b[:r].T.cpu()

    def full(self):
        r = self.rank
        return (self.a[:r].T @ self.b[:r]).cpu()

    def __repr__(self):
        return f"DevTT({self.n1}x{self.n2}, rank={self.rank}, cap={self.cap})"


def _ws(nbytes, device="cuda"):
    nbytes = max(int(nbytes), 256)
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def tt_round(x, tol, rank_cap, y=None, stream=None):
    _require_cuda()
    lib = C.load()
    if y is None:
        y = DevTT(x.n1, x.n2, rank_cap)
    ws = _ws(lib.tt_round_workspace_size(x.n1, x.n2, x.rank, rank_cap))
    xs, ys = x.struct(), y.struct()
    err = ctypes.c_double(0.0)
    C.check("tt_round", lib.tt_round(ctypes.byref(xs), tol, rank_cap, ctypes.byref(ys), ctypes.byref(err),
                                      ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
    y.rank = ys.rank
    return y, err.value


def tt_round_hadamard(x, z, tol, rank_cap, y=None, stream=None):
    _require_cuda()
    lib = C.load()
    if y is None:
        y = DevTT(x.n1, x.n2, rank_cap)
    ws = _ws(lib.tt_round_hadamard_workspace_size(x.n1, x.n2, x.rank, z.rank, rank_cap))
    xs, zs, ys = x.struct(), z.struct(), y.struct()
    C.check("tt_round_hadamard", lib.tt_round_hadamard(ctypes.byref(xs), ctypes.byref(zs), tol, rank_cap,
                                                       ctypes.byref(ys), ctypes.c_void_p(ws.data_ptr()),
                                                       ws.numel(), _stream_ptr(stream)))
    y.rank = ys.rank
    return y


def tt_cross(fn, inputs, x0, fparams, tol, rank_cap, n1, n2, kick=4, max_sweeps=10, seed=0, y=None,
             stream=None):
    _require_cuda()
    lib = C.load()
    if y is None:
        y = DevTT(n1, n2, rank_cap)
    rin = max(t.rank for t in list(inputs) + [x0])
    ws = _ws(lib.tt_cross_workspace_size(n1, n2, rin, rank_cap, kick) + 8 * n1 * n2 + (16 << 20))
    arr = (C.tt2 * len(inputs))(*[t.struct() for t in inputs])
    x0s, ys = x0.struct(), y.struct()
    prm = (ctypes.c_double * 4)(*(list(fparams) + [0.0] * (4 - len(fparams))))
    sw = ctypes.c_int32(0)
    C.check("tt_cross", lib.tt_cross(fn, arr, len(inputs), ctypes.byref(x0s), prm, tol, rank_cap, kick,
                                     max_sweeps, seed, ctypes.byref(ys), ctypes.byref(sw),
                                     ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
    y.rank = ys.rank
    return y, sw.value


def tt_maxvol(U, delta=1e-2, max_iter=200, stream=None):
    """Maximum-volume rows of the n x r FP64 CUDA tensor U: an int32 CUDA
    tensor of r row indices (tt_maxvol)."""
    _require_cuda()
    lib = C.load()
    n, r = U.shape
    Uc = U.t().contiguous()  # column-major n x r
    idx = torch.empty(r, dtype=torch.int32, device=U.device)
    ws = _ws(lib.tt_maxvol_workspace_size(n, r))
    C.check("tt_maxvol", lib.tt_maxvol(ctypes.c_void_p(Uc.data_ptr()), n, r, delta, max_iter,
                                       ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                       _stream_ptr(stream)))
    return idx


def tt_reciprocal(x, tol, rank_cap, max_iter=50, y=None, stream=None):
    _require_cuda()
    lib = C.load()
    if y is None:
        y = DevTT(x.n1, x.n2, rank_cap)
    ws = _ws(lib.tt_reciprocal_workspace_size(x.n1, x.n2, x.rank, rank_cap))
    xs, ys = x.struct(), y.struct()
    it = ctypes.c_int32(0)
    C.check("tt_reciprocal", lib.tt_reciprocal(ctypes.byref(xs), tol, rank_cap, max_iter, ctypes.byref(ys),
                                               ctypes.byref(it), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                               _stream_ptr(stream)))
    y.rank = ys.rank
    return y, it.value


def tt_recon_linear(x, direction, scheme, stream=None):
    _require_cuda()
    lib = C.load()
    nq = 2 if scheme == C.TT_UP3 else 3
    f1, f2 = (x.n1, nq * x.n2) if direction == 0 else (nq * x.n1, x.n2)
    qm, qp = DevTT(f1, f2, x.rank), DevTT(f1, f2, x.rank)
    xs, ms, ps = x.struct(), qm.struct(), qp.struct()
    C.check("tt_recon_linear", lib.tt_recon_linear(ctypes.byref(xs), direction, scheme, ctypes.byref(ms),
                                                   ctypes.byref(ps), _stream_ptr(stream)))
    qm.rank, qp.rank = ms.rank, ps.rank
    return qm, qp


def tt_contract(A, B, precision="fp64", split=True, alpha=1.0, beta=0.0, C=None, stream=None):
    """C = alpha A B + beta C for float64 CUDA tensors A (m x k), B (k x n)
    (any strides with unit row stride are re-laid out column-major here)."""
    _require_cuda()
    lib = C_.load()
    m, k = A.shape
    k2, n = B.shape
    if k2 != k:
        raise ValueError("inner dimensions differ")
    Ac = A.t().contiguous().t() if A.stride(0) != 1 else A
    Bc = B.t().contiguous().t() if B.stride(0) != 1 else B
    if C is None:
        C = torch.zeros((n, m), dtype=torch.float64, device=A.device).t()
    prec = C_.PRECISIONS[precision]
    ws = _ws(lib.tt_contract_workspace_size(prec, int(bool(split)), m, n, k))
    C_.check("tt_contract", lib.tt_contract(prec, int(bool(split)), m, n, k, alpha, ctypes.c_void_p(Ac.data_ptr()),
                                            Ac.stride(1), ctypes.c_void_p(Bc.data_ptr()), Bc.stride(1), beta,
                                            ctypes.c_void_p(C.data_ptr()), C.stride(1),
                                            ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
    return C


def launch_count():
    """Kernels launched by libttfv.so in this process so far."""
    return int(C.load().tt_launch_count())


def tile_shapes():
    """The TSQR tile shapes (leaf-row multiple, largest merge fan-in; 0 is the
    default fan-in) a solver can be switched to; shape 0 is the default."""
    lib = C.load()
    K = lib.tt_tile_shapes(None, None, 0)
    lm, fi = (ctypes.c_int32 * K)(), (ctypes.c_int32 * K)()
    lib.tt_tile_shapes(lm, fi, K)
    return [(lm[k], fi[k]) for k in range(K)]


class Solver:
    """tt_fv_init / tt_fv_stage / tt_fv_step / tt_fv_get over a torch workspace."""

    def __init__(self, q0, eqn, scheme, n, dt, tol, rank_cap, g=9.81, H=1.0, f=0.0, lx=1.0, ly=1.0,
                 kick=4, max_sweeps=10, max_iter=50, seed=0, precision="fp64", pivots="maxvol", stream=None,
                 eps_rule="fixed", c_eps=1.0, flux="products", forcing_waves=0, bc_x="periodic",
                 boundary_waves=0):
        _require_cuda()
        self.lib = C.load()
        self.p = C.tt_fv_params(C.EQNS[eqn], C.SCHEMES[scheme], n, n, lx, ly, g, H, f, dt, tol, rank_cap,
                                C.PRECISIONS[precision], C.PIVOTS[pivots], kick, max_sweeps, max_iter, seed,
                                C.EPS_RULES[eps_rule], c_eps, C.FLUXES[flux], forcing_waves, C.BCS[bc_x],
                                boundary_waves)
        nbytes = self.lib.tt_fv_workspace_size(ctypes.byref(self.p))
        if nbytes == 0:
            raise C.TTError("tt_fv_workspace_size", C.TT_ERR_ARG)
        self.ws = _ws(nbytes)
        self.stream = stream
        self.n, self.cap = n, rank_cap
        arr = (C.tt2 * 3)(*[q.struct() for q in q0])
        h = ctypes.c_void_p()
        C.check("tt_fv_init", self.lib.tt_fv_init(ctypes.byref(self.p), arr, ctypes.c_void_p(self.ws.data_ptr()),
                                                  self.ws.numel(), _stream_ptr(stream), ctypes.byref(h)))
        self.h = h

    def stage(self, k):
        C.check("tt_fv_stage", self.lib.tt_fv_stage(self.h, k))

    def step(self, n=1):
        C.check("tt_fv_step", self.lib.tt_fv_step(self.h, n))

    def get(self):
        out = [DevTT(self.n, self.n, self.cap) for _ in range(3)]
        arr = (C.tt2 * 3)(*[q.struct() for q in out])
        C.check("tt_fv_get", self.lib.tt_fv_get(self.h, arr))
        for q, s in zip(out, arr):
            q.rank = s.rank
        return out

    def set(self, q):
        arr = (C.tt2 * 3)(*[t.struct() for t in q])
        C.check("tt_fv_set", self.lib.tt_fv_set(self.h, arr))

    def set_forcing(self, waves, t0=0.0):
        """waves: (field, amp, kx, ky, omega, phase[, decay]) waves of the source."""
        arr = (C.tt_wave * max(1, len(waves)))(*[C.tt_wave(int(f), *map(float, rest)) for f, *rest in waves])
        C.check("tt_fv_set_forcing", self.lib.tt_fv_set_forcing(self.h, arr, len(waves), float(t0)))

    def set_boundary(self, waves, t0=0.0):
        """waves: (field, amp, kx, ky, omega, phase[, decay]) waves of the exact
        solution whose cell averages fill the x-boundary ghost cells."""
        arr = (C.tt_wave * max(1, len(waves)))(*[C.tt_wave(int(f), *map(float, rest)) for f, *rest in waves])
        C.check("tt_fv_set_boundary", self.lib.tt_fv_set_boundary(self.h, arr, len(waves), float(t0)))

    def stats(self):
        st = C.tt_fv_stats()
        C.check("tt_fv_stats_get", self.lib.tt_fv_stats_get(self.h, ctypes.byref(st)))
        return {k: (list(getattr(st, k)) if k in ("rank", "section_ms", "eps_u") else getattr(st, k))
                for k, _ in st._fields_}

    def profile(self, enable=True):
        C.check("tt_fv_profile", self.lib.tt_fv_profile(self.h, 1 if enable else 0))

    def set_tile_shape(self, shape):
        """Use TSQR tile shape `shape` (an index into tile_shapes())."""
        C.check("tt_fv_set_tile_shape", self.lib.tt_fv_set_tile_shape(self.h, shape))

    def kernel_profile(self, reset=False):
        arr = (C.tt_kernel_prof * len(C.TT_K_NAMES))()
        C.check("tt_fv_kernel_profile", self.lib.tt_fv_kernel_profile(self.h, arr, 1 if reset else 0))
        return {name: dict(ms=r.ms, flops=r.flops, bytes=r.bytes, launches=r.launches)
                for name, r in zip(C.TT_K_NAMES, arr)}

    def set_pivot_net(self, net):
        """Start every cross from `net`'s proposals (a PivotNet; None: maxvol start)."""
        self._net = net
        st = net.struct() if net is not None else None
        C.check("tt_fv_set_pivot_net", self.lib.tt_fv_set_pivot_net(self.h, ctypes.byref(st) if st else None))

    def record_pivots(self, enable=True):
        C.check("tt_fv_record_pivots", self.lib.tt_fv_record_pivots(self.h, 1 if enable else 0))

    def take_pivots(self):
        """Captured (features rows x 14, labels rows) as numpy float32 arrays."""
        import numpy as np
        rows = int(self.lib.tt_fv_pivot_rows(self.h))
        X = np.empty((rows, 14), dtype=np.float32)
        y = np.empty(rows, dtype=np.float32)
        C.check("tt_fv_pivot_take", self.lib.tt_fv_pivot_take(self.h, X.ctypes.data_as(ctypes.c_void_p),
                                                              y.ctypes.data_as(ctypes.c_void_p), rows))
        return X, y

    def close(self):
        if getattr(self, "h", None):
            self.lib.tt_fv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """tt_fv_batch_*: an ensemble of independent solver instances advanced
    together (one workspace, one stream per instance)."""

    def __init__(self, instances, precision="fp64", workers=8, inner_tasks=False, stream=None):
        """instances: list of (q0, params) with q0 = three DevTT and params a
        dict with eqn, scheme, n, dt, tol, rank_cap and optional g, H, f,
        kick, max_sweeps, max_iter, seed."""
        _require_cuda()
        self.lib = C.load()
        self.count = len(instances)
        P = (C.tt_fv_params * self.count)()
        Q = (C.tt2 * (3 * self.count))()
        self.shapes = []
        for i, (q0, d) in enumerate(instances):
            P[i] = C.tt_fv_params(C.EQNS[d["eqn"]], C.SCHEMES[d["scheme"]], d["n"], d["n"], 1.0, 1.0,
                                  d.get("g", 9.81), d.get("H", 1.0), d.get("f", 0.0), d["dt"], d["tol"],
                                  d["rank_cap"], C.PRECISIONS[precision], C.TT_PIVOT_MAXVOL, d.get("kick", 4),
                                  d.get("max_sweeps", 10), d.get("max_iter", 50), d.get("seed", 0))
            for c in range(3):
                Q[3 * i + c] = q0[c].struct()
            self.shapes.append((d["n"], d["rank_cap"]))
        nbytes = self.lib.tt_fv_batch_workspace_size(P, self.count)
        if nbytes == 0:
            raise C.TTError("tt_fv_batch_workspace_size", C.TT_ERR_ARG)
        self.ws = _ws(nbytes)
        h = ctypes.c_void_p()
        C.check("tt_fv_batch_init", self.lib.tt_fv_batch_init(P, self.count, Q, ctypes.c_void_p(self.ws.data_ptr()),
                                                              self.ws.numel(), _stream_ptr(stream), ctypes.byref(h)))
        self.h = h
        self.configure(workers, inner_tasks)

    def configure(self, workers, inner_tasks=False):
        C.check("tt_fv_batch_configure", self.lib.tt_fv_batch_configure(self.h, workers, 1 if inner_tasks else 0))

    def step(self, n=1):
        C.check("tt_fv_batch_step", self.lib.tt_fv_batch_step(self.h, n))

    def tune(self, workers=(4, 8, 16, 32), steps_per_trial=1, with_rates=False):
        """Autotune (worker count, inner tasks) on real steps; returns the
        chosen pair (and, with_rates, {(workers, inner): cell updates/s})."""
        arr = (ctypes.c_int32 * len(workers))(*workers)
        bw, bi = ctypes.c_int32(0), ctypes.c_int32(0)
        rates = (ctypes.c_double * (2 * len(workers)))()
        C.check("tt_fv_batch_tune", self.lib.tt_fv_batch_tune(self.h, arr, len(workers), steps_per_trial,
                                                              ctypes.byref(bw), ctypes.byref(bi), rates))
        if with_rates:
            tab = {(w, bool(i)): rates[2 * c + i] for c, w in enumerate(workers) for i in (0, 1)}
            return (bw.value, bool(bi.value)), tab
        return bw.value, bool(bi.value)

    def tune_tiles(self, steps_per_trial=1, rounds=1):
        """Autotune each instance's TSQR tile shape on real steps (every shape
        of tile_shapes() timed rounds x steps_per_trial steps); returns the
        per-instance shape indices and {shape: batch cell updates/s}."""
        K = self.lib.tt_tile_shapes(None, None, 0)
        n = len(self.shapes)
        out = (ctypes.c_int32 * n)()
        rates = (ctypes.c_double * K)()
        C.check("tt_fv_batch_tune_tiles",
                self.lib.tt_fv_batch_tune_tiles(self.h, steps_per_trial, rounds, out, rates))
        return list(out), {k: rates[k] for k in range(K)}

    def get(self, i):
        n, cap = self.shapes[i]
        out = [DevTT(n, n, cap) for _ in range(3)]
        arr = (C.tt2 * 3)(*[q.struct() for q in out])
        C.check("tt_fv_batch_get", self.lib.tt_fv_batch_get(self.h, i, arr))
        for q, s in zip(out, arr):
            q.rank = s.rank
        return out

    def stats(self, i):
        st = C.tt_fv_stats()
        C.check("tt_fv_batch_stats_get", self.lib.tt_fv_batch_stats_get(self.h, i, ctypes.byref(st)))
        return {k: (list(getattr(st, k)) if k in ("rank", "section_ms", "eps_u") else getattr(st, k))
                for k, _ in st._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.tt_fv_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PivotNet:
    """Device parameters of the learned-pivot network (tt_mlp) with Adam
    moments; weights as float32 CUDA tensors (W1 14x256, W2 256x256
    row-major, b1, b2, w3 of 256, b3 of 1)."""

    NAMES = ("W1", "b1", "W2", "b2", "w3", "b3")
    SHAPES = {"W1": (14, 256), "b1": (256,), "W2": (256, 256), "b2": (256,), "w3": (256,), "b3": (1,)}

    def __init__(self, params=None, device="cuda"):
        _require_cuda()
        self.lib = C.load()
        self.p = {k: torch.zeros(self.SHAPES[k], dtype=torch.float32, device=device) for k in self.NAMES}
        if params is not None:
            self.load(params)
        self.g = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.m1 = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.m2 = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.t = 0

    @classmethod
    def shipped(cls, device="cuda"):
        """The network trained by train_pivots.py on plain-cross pivots of
        seeded 128^2 and 256^2 WENO5 runs (pivot_net.npz beside this file)."""
        import os
        import numpy as np
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pivot_net.npz")
        with np.load(path) as f:
            return cls({k: f[k] for k in cls.NAMES}, device=device)

    def load(self, params):
        for k in self.NAMES:
            self.p[k].copy_(torch.as_tensor(params[k], dtype=torch.float32).reshape(self.SHAPES[k]))

    def host(self):
        return {k: v.cpu().numpy().copy() for k, v in self.p.items()}

    @staticmethod
    def _struct(d):
        return C.tt_mlp(*[d[k].data_ptr() for k in PivotNet.NAMES])

    def struct(self):
        return self._struct(self.p)

    def forward(self, X, stream=None):
        """Scores of the rows of X (m x 14 float32 CUDA tensor)."""
        Xc = X.t().contiguous()  # column-major m x 14
        m = X.shape[0]
        s = torch.empty(m, dtype=torch.float32, device=X.device)
        ws = _ws(self.lib.tt_mlp_workspace_size(m, 1))
        net = self.struct()
        C.check("tt_mlp_forward", self.lib.tt_mlp_forward(ctypes.byref(net), ctypes.c_void_p(Xc.data_ptr()), m,
                                                          ctypes.c_void_p(s.data_ptr()),
                                                          ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                                          _stream_ptr(stream)))
        return s

    def grad(self, X, y, stream=None):
        """Gradients (into self.g) and the mean logistic loss of rows X, labels y."""
        Xc = X.t().contiguous()
        m = X.shape[0]
        yc = y.to(torch.float32).contiguous()
        loss = torch.zeros(1, dtype=torch.float64, device=X.device)
        ws = _ws(self.lib.tt_mlp_workspace_size(m, 1))
        net, g = self.struct(), self._struct(self.g)
        C.check("tt_mlp_grad", self.lib.tt_mlp_grad(ctypes.byref(net), ctypes.c_void_p(Xc.data_ptr()),
                                                    ctypes.c_void_p(yc.data_ptr()), m, ctypes.byref(g),
                                                    ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                                    ws.numel(), _stream_ptr(stream)))
        return loss

    def adam_step(self, lr, stream=None):
        self.t += 1
        net, g, m1, m2 = self.struct(), self._struct(self.g), self._struct(self.m1), self._struct(self.m2)
        C.check("tt_mlp_adam", self.lib.tt_mlp_adam(ctypes.byref(net), ctypes.byref(g), ctypes.byref(m1),
                                                    ctypes.byref(m2), self.t, lr, _stream_ptr(stream)))

    def train_step(self, X, y, lr, stream=None):
        loss = self.grad(X, y, stream)
        self.adam_step(lr, stream)
        return loss


def tt_mlp_features(x0, prev=(), stream=None):
    """Index features (n2 x 14 float32 CUDA tensor, row-major view) of x0's
    column mode; prev: the site's previous converged pivot indices."""
    _require_cuda()
    lib = C.load()
    Xc = torch.empty((14, x0.n2), dtype=torch.float32, device="cuda")  # column-major n2 x 14
    pv = torch.tensor(list(prev) or [0], dtype=torch.int32, device="cuda")
    ws = _ws(lib.tt_mlp_workspace_size(x0.n2, x0.rank))
    xs = x0.struct()
    C.check("tt_mlp_features", lib.tt_mlp_features(ctypes.byref(xs), ctypes.c_void_p(pv.data_ptr()), len(prev),
                                                   ctypes.c_void_p(Xc.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                                   ws.numel(), _stream_ptr(stream)))
    return Xc.t()


def tt_mlp_topk(s, k, stream=None):
    """The k highest scores' indices (ascending; ties to the smaller index)."""
    _require_cuda()
    lib = C.load()
    m = s.shape[0]
    idx = torch.empty(k, dtype=torch.int32, device=s.device)
    ws = _ws(lib.tt_mlp_workspace_size(m, 1))
    sc = s.to(torch.float32).contiguous()
    C.check("tt_mlp_topk", lib.tt_mlp_topk(ctypes.c_void_p(sc.data_ptr()), m, k, ctypes.c_void_p(idx.data_ptr()),
                                           ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
    return idx
