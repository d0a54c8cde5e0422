"""Python binding of libtatrg (GB300 Triad-ATRG).  Argument marshalling only: every step
of the coarse-graining runs in the library's CUDA kernels.  PyTorch supplies device memory
and streams for the building-block calls.

The library must have been built (``python -m paper_2412_14104_gb300.build``); importing
the binding without it raises, there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtatrg.so")

FP64, TF32X3, BF16X3, BF16X6, OZAKI = 0, 1, 2, 3, 4
ATRG, TRIAD = 0, 1
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENUMERIC", 5: "ETIMEOUT",
           6: "ESTATE", 7: "ENOTIMPL"}


class TatrgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_STATUS.get(code, code), msg))
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("chi", ctypes.c_int), ("r", ctypes.c_int), ("q", ctypes.c_int),
                ("method", ctypes.c_int), ("precision", ctypes.c_int),
                ("seed", ctypes.c_ulonglong), ("checkpoint_every", ctypes.c_int),
                ("split_from_step", ctypes.c_int), ("split_stages", ctypes.c_int),
                ("profile", ctypes.c_int), ("sweep_workers", ctypes.c_int),
                ("early_precision", ctypes.c_int), ("late_from_step", ctypes.c_int)]


class StepInfo(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int), ("dims", ctypes.c_int * 5), ("swap_exact", ctypes.c_int),
                ("lnc", ctypes.c_double), ("flops", ctypes.c_double * 5),
                ("ms", ctypes.c_double * 5), ("swap_gap", ctypes.c_double),
                ("tc_launches", ctypes.c_int), ("kernel_launches", ctypes.c_int),
                ("tc_ms", ctypes.c_double), ("tc_flops", ctypes.c_double),
                ("partial_lnz", ctypes.c_double)]


class Contraction(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64 * 4) for n in
                ("m_ext", "m_sA", "m_sC", "n_ext", "n_sB", "n_sC", "k_ext", "k_sA", "k_sB")] + \
               [("alpha", ctypes.c_double), ("beta", ctypes.c_double)]


_lib = None


def lib():
    """The loaded libtatrg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtatrg.so is not built; run python -m paper_2412_14104_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        P, D, I, I64, U64, U32 = (ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                  ctypes.c_int64, ctypes.c_ulonglong, ctypes.c_uint32)
        sig = {
            "tatrg_create": [ctypes.POINTER(Params), P, ctypes.POINTER(P)],
            "tatrg_init_ising": [P, ctypes.c_double, ctypes.c_double, I],
            "tatrg_rg_step": [P, I],
            "tatrg_lnZ": [P, D],
            "tatrg_grad": [P, D, D, D],
            "tatrg_sweep": [P, D, I, ctypes.c_double, I, I, D],
            "tatrg_sweep_observables": [P, D, I, ctypes.c_double, I, I, D, D],
            "tatrg_order_parameter": [P, I, D],
            "tatrg_spectrum": [P, I, D, ctypes.POINTER(I)],
            "tatrg_get_state": [P, ctypes.POINTER(I), ctypes.POINTER(I), D, D, D],
            "tatrg_set_state": [P, I, ctypes.POINTER(I), D, D, D, I, ctypes.c_double],
            "tatrg_last_step_info": [P, ctypes.POINTER(StepInfo)],
            "tatrg_gaussian": [U64, U32, U32, I64, I64, P, P],
            "tatrg_contract": [ctypes.POINTER(Contraction), I, P, P, P, P],
            "tatrg_contract_sketch": [ctypes.POINTER(Contraction), I, P, U64, U32, U32, P, P],
            "tatrg_orth": [I, I64, I64, P, P, P, ctypes.POINTER(I), P],
            "tatrg_svd": [I64, I64, P, P, P, P, P],
            "tatrg_svd_noalloc": [I64, I64, P, P, P, P, P],
            "tatrg_philox_words": [U64, U32, U32, U64, I64, P, P],
            "tatrg_set_barrier_limit_ns": [ctypes.c_longlong],
            "tatrg_set_cta_pairs": [I],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.tatrg_last_error.argtypes = [P]
        L.tatrg_last_error.restype = ctypes.c_char_p
        L.tatrg_destroy.argtypes = [P]
        L.tatrg_destroy.restype = None
        _lib = L
    return _lib


def _check(code, ctx=None):
    if code != 0:
        msg = lib().tatrg_last_error(ctx)
        raise TatrgError(code, msg.decode() if msg else "")


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _reach(modes, which):
    """Elements a mode list can address from its base pointer: 1 + the largest offset
    sum (ext - 1) * stride over the modes, with the stride taken from position `which`
    of each (ext, stride, stride) triple; 0 when an extent is 0."""
    top = 0
    for m in modes:
        e, st = int(m[0]), int(m[which])
        if e < 0 or st < 0:
            raise TatrgError(1, "mode extents and strides must be non-negative, got %r" % (tuple(m),))
        if e == 0:
            return 0
        top += (e - 1) * st
    return top + 1


def _device_ptrs(*specs):
    """Device pointers of the caller's tensors, each spec (tensor, elements, name[, dtypes]),
    after checking that every tensor can hold what the call will address: dtype float64
    (unless the spec names others), contiguous, at least that many elements, then a CUDA
    tensor on the current device.  The library reaches caller memory only through these
    pointers and the call's sizes, so a mismatch is reported here (EINVAL) instead of
    becoming an out-of-range access on the GPU."""
    import torch
    for spec in specs:
        t, nelem, what = spec[:3]
        dtypes = spec[3] if len(spec) > 3 else (torch.float64,)
        if not isinstance(t, torch.Tensor):
            raise TatrgError(1, "%s must be a torch tensor" % what)
        if t.dtype not in dtypes:
            raise TatrgError(1, "%s must have dtype %s, got %s" % (what, "/".join(map(str, dtypes)), t.dtype))
        if not t.is_contiguous():
            raise TatrgError(1, "%s must be contiguous" % what)
        if t.numel() < nelem:
            raise TatrgError(1, "%s holds %d elements, the call addresses %d" % (what, t.numel(), nelem))
    out = []
    for t, _, what, *_ in specs:
        if not t.is_cuda:
            raise TatrgError(1, "%s must be a CUDA tensor" % what)
        if t.device.index != torch.cuda.current_device():
            raise TatrgError(1, "%s is on cuda:%d, the current device is cuda:%d"
                             % (what, t.device.index, torch.cuda.current_device()))
        out.append(ctypes.c_void_p(t.data_ptr()))
    return out


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """One RG run on the current CUDA device (tatrg_ctx)."""

    def __init__(self, chi, r, q=2, method=TRIAD, precision=FP64, seed=0, split_from_step=0,
                 split_stages=0, profile=0, sweep_workers=0, stream=None, early_precision=0,
                 late_from_step=0):
        self.params = Params(chi, r, q, method, precision, seed, 4, split_from_step, split_stages,
                             profile, sweep_workers, early_precision, late_from_step)
        h = ctypes.c_void_p()
        _check(lib().tatrg_create(ctypes.byref(self.params), _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    def close(self):
        if self._h:
            lib().tatrg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_ising(self, beta, h, d):
        _check(lib().tatrg_init_ising(self._h, beta, h, d), self._h)
        return self

    def rg_step(self, n=1):
        _check(lib().tatrg_rg_step(self._h, n), self._h)
        return self

    def lnZ(self):
        out = ctypes.c_double()
        _check(lib().tatrg_lnZ(self._h, ctypes.byref(out)), self._h)
        return out.value

    def grad(self, second=False):
        """(dlnZ/dbeta, dlnZ/dh, d2lnZ/dbeta2 or None) of the run so far, per site."""
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().tatrg_grad(self._h, ctypes.byref(a), ctypes.byref(b),
                                ctypes.byref(c) if second else None), self._h)
        return a.value, b.value, (c.value if second else None)

    def sweep(self, betas, h, d, nsteps):
        b = np.ascontiguousarray(betas, dtype=np.float64)
        out = np.empty_like(b)
        _check(lib().tatrg_sweep(self._h, _dptr(b), b.size, h, d, nsteps, _dptr(out)), self._h)
        return out

    def sweep_observables(self, betas, h, d, nsteps):
        """(ln Z / V of every temperature run, X^(m) at leg d - 1 after every step as an
        array of shape (len(betas), nsteps))."""
        b = np.ascontiguousarray(betas, dtype=np.float64)
        z, x = np.empty_like(b), np.empty((b.size, nsteps))
        _check(lib().tatrg_sweep_observables(self._h, _dptr(b), b.size, h, d, nsteps, _dptr(z),
                                             _dptr(x)), self._h)
        return z, x

    def order_parameter(self, leg):
        out = ctypes.c_double()
        _check(lib().tatrg_order_parameter(self._h, leg, ctypes.byref(out)), self._h)
        return out.value

    def spectrum(self, kind):
        n = ctypes.c_int(0)
        _check(lib().tatrg_spectrum(self._h, kind, None, ctypes.byref(n)), self._h)
        out = np.empty(max(n.value, 1))
        _check(lib().tatrg_spectrum(self._h, kind, _dptr(out), ctypes.byref(n)), self._h)
        return out[:n.value]

    def get_state(self):
        d = ctypes.c_int()
        dims = (ctypes.c_int * 5)()
        _check(lib().tatrg_get_state(self._h, ctypes.byref(d), dims, None, None, None), self._h)
        dd = d.value
        D = [dims[i] for i in range(dd)]
        Da = dims[dd]
        A = np.empty(tuple(D) + (Da,))
        B = np.empty((Da,) + tuple(D))
        s = np.empty(Da)
        _check(lib().tatrg_get_state(self._h, ctypes.byref(d), dims, _dptr(A), _dptr(s), _dptr(B)), self._h)
        return A, s, B

    def set_state(self, A, s, B, step, partial_lnz):
        A, s, B = np.asarray(A), np.asarray(s), np.asarray(B)
        d = A.ndim - 1
        if not 2 <= d <= 4 or s.ndim != 1 or A.shape[d] != s.size or B.shape != (s.size,) + A.shape[:d]:
            raise TatrgError(1, "set_state: need A (D_0..D_{d-1}, Da), s (Da,), B (Da, D_0..D_{d-1}) "
                                "with 2 <= d <= 4; got %s, %s, %s" % (A.shape, s.shape, B.shape))
        dims = (ctypes.c_int * 5)(*(list(A.shape[:d]) + [s.size] + [0] * (4 - d)))
        A = np.ascontiguousarray(A, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
        s = np.ascontiguousarray(s, dtype=np.float64)
        _check(lib().tatrg_set_state(self._h, d, dims, _dptr(A), _dptr(s), _dptr(B), step,
                                     partial_lnz), self._h)
        return self

    def step_info(self):
        info = StepInfo()
        _check(lib().tatrg_last_step_info(self._h, ctypes.byref(info)), self._h)
        return info


# --- building blocks on torch CUDA tensors --------------------------------------------

def gaussian(seed, stream_id, rows, cols, out, replica=0, stream=None):
    (po,) = _device_ptrs((out, max(rows, 0) * max(cols, 0), "out"))
    _check(lib().tatrg_gaussian(seed, stream_id, replica, rows, cols, po, _stream_ptr(stream)))
    return out


def _contraction(m, n, k, alpha, beta):
    c = Contraction()
    for name, modes in (("m", m), ("n", n), ("k", k)):
        assert len(modes) <= 4
        full = list(modes) + [(1, 0, 0)] * (4 - len(modes))
        s1, s2 = {"m": ("m_sA", "m_sC"), "n": ("n_sB", "n_sC"), "k": ("k_sA", "k_sB")}[name]
        for i, (e, a, b) in enumerate(full):
            getattr(c, name + "_ext")[i] = e
            getattr(c, s1)[i] = a
            getattr(c, s2)[i] = b
    c.alpha, c.beta = alpha, beta
    return c


def _operand_ptrs(m, n, k, A, B, C):
    """Checked pointers of a contraction's operands (B may be None: a generated sketch).
    A is addressed through the m and k strides in A, B through n and k strides in B, C
    through the m and n strides in C; nothing is read or written when M or N is 0."""
    if _reach(m, 1) == 0 or _reach(n, 1) == 0:
        need_a = need_b = need_c = 0
    else:
        kk = _reach(k, 1) > 0
        need_a = _reach(m, 1) + _reach(k, 1) - 1 if kk else 0
        need_b = _reach(n, 1) + _reach(k, 2) - 1 if kk else 0
        need_c = _reach(m, 2) + _reach(n, 2) - 1
    if B is None:
        pa, pc = _device_ptrs((A, need_a, "A"), (C, need_c, "C"))
        return pa, None, pc
    return _device_ptrs((A, need_a, "A"), (B, need_b, "B"), (C, need_c, "C"))


def contract_sketch(m, n, k, A, seed, stream_id, C, replica=0, alpha=1.0, beta=0.0,
                    precision=TF32X3, stream=None):
    """contract() with B the Gaussian sketch (seed, stream_id, replica) generated in the
    tensor-core operand packer instead of read from memory (split precisions only)."""
    c = _contraction(m, n, k, alpha, beta)
    pa, _, pc = _operand_ptrs(m, n, k, A, None, C)
    _check(lib().tatrg_contract_sketch(ctypes.byref(c), precision, pa, seed, stream_id, replica, pc,
                                       _stream_ptr(stream)))
    return C


def contract(m, n, k, A, B, C, alpha=1.0, beta=0.0, precision=FP64, stream=None):
    """C[m, n] = alpha sum_k A[m, k] B[k, n] + beta C; m = [(ext, strideA, strideC), ...],
    n = [(ext, strideB, strideC), ...], k = [(ext, strideA, strideB), ...] (outermost first)."""
    c = _contraction(m, n, k, alpha, beta)
    pa, pb, pc = _operand_ptrs(m, n, k, A, B, C)
    _check(lib().tatrg_contract(ctypes.byref(c), precision, pa, pb, pc, _stream_ptr(stream)))
    return C


def orth(Y, Q, R, precision=FP64, stream=None):
    m, n = Y.shape
    k = ctypes.c_int()
    py, pq, pr = _device_ptrs((Y, m * n, "Y"), (Q, m * n, "Q"), (R, n * n, "R"))
    _check(lib().tatrg_orth(precision, m, n, py, pq, pr, ctypes.byref(k), _stream_ptr(stream)))
    return k.value


def _svd_ptrs(A, U, S, V):
    m, n = A.shape
    return (m, n, *_device_ptrs((A, m * n, "A"), (U, m * n, "U"), (S, n, "S"), (V, n * n, "V")))


def svd(A, U, S, V, stream=None):
    _check(lib().tatrg_svd(*_svd_ptrs(A, U, S, V), _stream_ptr(stream)))


def svd_noalloc(A, U, S, V, stream=None):
    """tatrg_svd_noalloc: the same SVD with its workspace in the library's fixed device
    array instead of allocated memory (for callers that cannot allocate)."""
    _check(lib().tatrg_svd_noalloc(*_svd_ptrs(A, U, S, V), _stream_ptr(stream)))


def philox_words(seed, stream_id, first, npairs, out, replica=0, stream=None):
    """Raw Philox4x32-10 words of counter blocks first .. first + npairs - 1 into the int32
    CUDA tensor `out` (4 words per block)."""
    import torch
    words = tuple(t for t in (torch.int32, getattr(torch, "uint32", None)) if t is not None)
    (po,) = _device_ptrs((out, 4 * max(npairs, 0), "out", words))
    _check(lib().tatrg_philox_words(seed, stream_id, replica, first, npairs, po, _stream_ptr(stream)))
    return out


def set_barrier_limit_ns(limit_ns):
    """Time limit of the cooperative Jacobi SVD's grid-barrier waits on the current device."""
    _check(lib().tatrg_set_barrier_limit_ns(int(limit_ns)))


def set_cta_pairs(mode):
    """Tile form of the split-precision contractions: 0 autotuned, 1 CTA pairs, 2 multicast
    clusters wherever they apply (M >= 1024), -1 single CTAs only."""
    _check(lib().tatrg_set_cta_pairs(int(mode)))


def lnz_function(chi, r, q=2, method=TRIAD, precision=FP64, seed=0, d=4, nsteps=8):
    """ln Z / V of a run as a torch.autograd.Function of the scalar tensors (beta, h).

    The forward call runs the RG steps and the tangent passes of tatrg_grad; backward
    returns grad_output times dlnZ/dbeta and dlnZ/dh.  Both inputs are 0-d float64 tensors.
    """
    import torch

    class _LnZ(torch.autograd.Function):
        @staticmethod
        def forward(fctx, beta, h):
            ctx = Context(chi, r, q, method=method, precision=precision, seed=seed)
            ctx.init_ising(float(beta), float(h), d).rg_step(nsteps)
            lnz = ctx.lnZ()
            gb, gh, _ = ctx.grad()
            fctx.save_for_backward(torch.tensor([gb, gh], dtype=torch.float64))
            return torch.tensor(lnz, dtype=torch.float64)

        @staticmethod
        def backward(fctx, grad_out):
            (g,) = fctx.saved_tensors
            return grad_out * g[0], grad_out * g[1]

    return _LnZ.apply
