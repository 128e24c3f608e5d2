"""Python front end of the CUDA TT finite-volume library.

Device memory comes from PyTorch (cores, workspaces); the functions here only
marshal arguments to the C ABI (include/tt_fv.h) -- the names match it.
"""
import ctypes

import torch

from . import capi as C


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


def launch_count():
    """Kernels launched by libttfv.so in this process so far."""
    return int(C.load().tt_launch_count())


class Solver:
    """tt_fv_init / tt_fv_stage / tt_fv_step / tt_fv_get over a torch workspace."""

    def __init__(self, q0, eqn, scheme, n, dt, tol, rank_cap, g=9.81, H=1.0, f=0.0, lx=1.0, ly=1.0,
                 kick=4, max_sweeps=10, max_iter=50, seed=0, stream=None):
        _require_cuda()
        self.lib = C.load()
        self.p = C.tt_fv_params(C.EQNS[eqn], C.SCHEMES[scheme], n, n, lx, ly, g, H, f, dt, tol, rank_cap,
                                C.TT_FP64, C.TT_PIVOT_MAXVOL, kick, max_sweeps, max_iter, seed)
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

    def stats(self):
        st = C.tt_fv_stats()
        C.check("tt_fv_stats_get", self.lib.tt_fv_stats_get(self.h, ctypes.byref(st)))
        return {k: (list(getattr(st, k)) if k in ("rank", "section_ms") else getattr(st, k))
                for k, _ in st._fields_}

    def profile(self, enable=True):
        C.check("tt_fv_profile", self.lib.tt_fv_profile(self.h, 1 if enable else 0))

    def kernel_profile(self, reset=False):
        arr = (C.tt_kernel_prof * len(C.TT_K_NAMES))()
        C.check("tt_fv_kernel_profile", self.lib.tt_fv_kernel_profile(self.h, arr, 1 if reset else 0))
        return {name: dict(ms=r.ms, flops=r.flops, bytes=r.bytes, launches=r.launches)
                for name, r in zip(C.TT_K_NAMES, arr)}

    def close(self):
        if getattr(self, "h", None):
            self.lib.tt_fv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
