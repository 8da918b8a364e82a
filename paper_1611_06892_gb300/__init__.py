"""Python binding of the GB300 tiled band-bidiagonalization library (``libbidiag.so``, C ABI in
``include/bidiag.h``).

Argument marshalling only: every step of the reduction runs in the library's CUDA kernels; PyTorch
provides device memory and streams.  The library must have been built (``build.build()``); importing
the binding without it raises immediately - there is no CPU fallback.

Low-level functions carry the C names (``bidiag_create``, ``bidiag_band``, ...); ``Handle`` and
``Result`` wrap them for torch tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbidiag.so")

FLATTS, FLATTT, GREEDY, AUTO = 0, 1, 2, 3
TREES = {"flatts": FLATTS, "flattt": FLATTT, "greedy": GREEDY, "auto": AUTO}
BIDIAG, RBIDIAG, AUTO_VARIANT, THREESTEP = 0, 1, 2, 3
VARIANTS = {"bidiag": BIDIAG, "rbidiag": RBIDIAG, "auto": AUTO_VARIANT, "threestep": THREESTEP}


def threestep_split(s):
    """Variant code of the three-step reduction with s BiDiag steps before the switch (Sec. 4.5)."""
    return 4 + s
OK, ERR_CUDA, ERR_NOMEM, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_SCRATCH = 0, 1, 2, 3, 4, 5
NOALLOC_SCRATCH_BYTES = 8 << 20
OPT_WAIT_LIMIT_NS, OPT_AUTO_RESOURCES, OPT_DEBUG_UNSET_DEP, OPT_STRIP, OPT_TIMING, OPT_TRACE = 1, 2, 3, 4, 5, 6
OPT_F32_UPDATES = 7
OPT_F32_SCALARS = 8
OPT_WINDOW = 9
OPT_PRIORITY = 10

_lib = None


class BidiagError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bidiag error {code}: {msg}")
        self.code = code


class Reflectors(ctypes.Structure):
    _fields_ = [("tiles", ctypes.c_void_p), ("tiles2", ctypes.c_void_p), ("T", ctypes.c_void_p),
                ("tslot", ctypes.POINTER(ctypes.c_int32)), ("ntasks", ctypes.c_int64),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nb", ctypes.c_int32), ("ib", ctypes.c_int32),
                ("p", ctypes.c_int32), ("q", ctypes.c_int32), ("npanels", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("elem_bytes", ctypes.c_int32), ("tree", ctypes.c_int32)]


def load_library(path=LIB_PATH):
    """Loads libbidiag.so (raises if it is missing: build it with paper_1611_06892_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run `python -m paper_1611_06892_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    vp, i64, i32, cint = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "bidiag_create": (cint, [P(vp), cint, vp]),
        "bidiag_set_option": (cint, [vp, cint, i64]),
        "bidiag_band": (cint, [vp, i64, i64, vp, i64, cint, cint, cint, cint, P(vp)]),
        "bidiag_band_host": (cint, [vp, i64, i64, vp, i64, cint, cint, cint, cint, vp, i64, P(vp)]),
        "bidiag_band_f32": (cint, [vp, i64, i64, vp, i64, cint, cint, cint, cint, P(vp)]),
        "bidiag_band_batched": (cint, [vp, i64, P(i64), P(i64), P(vp), P(i64), P(cint), P(cint), P(cint), P(cint),
                                       P(vp)]),
        "bidiag_band_batched_f32": (cint, [vp, i64, P(i64), P(i64), P(vp), P(i64), P(cint), P(cint), P(cint),
                                           P(cint), P(vp)]),
        "bidiag_autotune": (cint, [i64, i64, cint, cint, P(cint), P(cint), P(cint), P(cint)]),
        "bidiag_result_band_f32": (cint, [vp, P(vp), P(i64), P(i64), P(cint)]),
        "bidiag_apply_q_f32": (cint, [vp, vp, cint, i64, vp, i64]),
        "bidiag_apply_p_f32": (cint, [vp, vp, cint, i64, vp, i64]),
        "bidiag_band_noalloc": (cint, [i64, i64, vp, i64, cint, cint, cint, cint, vp, i64, vp]),
        "bidiag_band_backward": (cint, [vp, vp, vp, i64, vp, i64, vp, i64]),
        "bidiag_band_backward_f32": (cint, [vp, vp, vp, i64, vp, i64, vp, i64]),
        "bidiag_result_band": (cint, [vp, P(vp), P(i64), P(i64), P(cint)]),
        "bidiag_result_tasks": (cint, [vp, P(P(i32)), P(i64)]),
        "bidiag_result_reflectors": (cint, [vp, P(Reflectors)]),
        "bidiag_apply_q": (cint, [vp, vp, cint, i64, vp, i64]),
        "bidiag_apply_p": (cint, [vp, vp, cint, i64, vp, i64]),
        "bidiag_sync": (cint, [vp]),
        "bidiag_last_exec_ms": (cint, [vp, P(ctypes.c_float)]),
        "bidiag_trace": (cint, [vp, P(i64), i64, P(i64)]),
        "bidiag_backward_workspace": (cint, [vp, vp, P(i64)]),
        "bidiag_trace_program": (cint, [vp, P(i32), i64, P(i64), P(i32), i64, P(i64)]),
        "bidiag_measure_fp64_peaks": (cint, [cint, vp, P(ctypes.c_double), P(ctypes.c_double)]),
        "bidiag_last_error": (ctypes.c_char_p, [vp]),
        "bidiag_result_free": (cint, [vp]),
        "bidiag_destroy": (cint, [vp]),
        "bidiag_plan_eliminations": (cint, [i64, i64, cint, cint, i64, P(i32), i64, P(i64)]),
        "bidiag_plan_tasks": (cint, [i64, i64, cint, cint, i64, P(i32), P(i32), i64, P(i64), P(i64)]),
        "bidiag_plan_choose_variant": (cint, [i64, i64, cint, i64, P(cint), P(i64), P(i64)]),
        "bidiag_plan_best_split": (cint, [i64, i64, cint, i64, P(cint), P(i64)]),
        "bidiag_plan_program": (cint, [i64, i64, cint, cint, cint, cint, i64, cint, P(i32), i64, P(i64), P(i32),
                                       i64, P(i64), P(i32)]),
        "bidiag_plan_backward": (cint, [i64, i64, cint, cint, cint, cint, i64, cint, P(i32), P(i32), i64, P(i64),
                                        P(i32), i64, P(i64), P(i64), i64, P(i64), P(i32), i64, P(i64), P(i32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(h, rc):
    if rc != 0:
        msg = load_library().bidiag_last_error(h).decode() if h else ""
        raise BidiagError(rc, msg)


# ---- thin wrappers with the C names ------------------------------------------------------------
def bidiag_create(device=0, stream=None):
    h = ctypes.c_void_p()
    _check(None, load_library().bidiag_create(ctypes.byref(h), device, stream))
    return h


def bidiag_set_option(h, option, value):
    _check(h, load_library().bidiag_set_option(h, option, value))


def bidiag_band(h, m, n, d_A, lda, nb, ib, tree, variant):
    r = ctypes.c_void_p()
    _check(h, load_library().bidiag_band(h, m, n, d_A, lda, nb, ib, tree, variant, ctypes.byref(r)))
    return r


def bidiag_band_f32(h, m, n, d_A, lda, nb, ib, tree, variant):
    r = ctypes.c_void_p()
    _check(h, load_library().bidiag_band_f32(h, m, n, d_A, lda, nb, ib, tree, variant, ctypes.byref(r)))
    return r


def bidiag_autotune(m, n, nsm, elem_bytes=8):
    """(nb, ib, tree, variant) the batched form's autotuner picks for an m x n matrix (FP64 storage:
    elem_bytes 8, FP32: 4)."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(None, load_library().bidiag_autotune(m, n, nsm, elem_bytes, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def bidiag_band_host(h, m, n, h_A, lda, nb, ib, tree, variant, h_ab, ldab, keep=False):
    r = ctypes.c_void_p()
    _check(h, load_library().bidiag_band_host(h, m, n, h_A, lda, nb, ib, tree, variant, h_ab, ldab,
                                              ctypes.byref(r) if keep else None))
    return r if keep else None


def bidiag_band_noalloc(m, n, d_A, lda, nb, ib, tree, variant, d_ab, ldab, stream=None):
    """Reduction that allocates no device memory (fixed static scratch); returns the status code."""
    return load_library().bidiag_band_noalloc(m, n, d_A, lda, nb, ib, tree, variant, d_ab, ldab, stream)


def bidiag_measure_fp64_peaks(device=0, stream=None):
    """Measured FP64 rates of the GPU (GFLOP/s): (DFMA loop, mma.sync m8n8k4 f64 loop)."""
    fma, mma = ctypes.c_double(), ctypes.c_double()
    rc = load_library().bidiag_measure_fp64_peaks(device, stream, ctypes.byref(fma), ctypes.byref(mma))
    if rc != OK:
        raise BidiagError(rc, "bidiag_measure_fp64_peaks failed")
    return fma.value, mma.value


def bidiag_sync(h):
    _check(h, load_library().bidiag_sync(h))


def bidiag_last_exec_ms(h):
    ms = ctypes.c_float()
    _check(h, load_library().bidiag_last_exec_ms(h, ctypes.byref(ms)))
    return ms.value


def bidiag_apply_q(h, r, trans, ncols, d_C, ldc):
    _check(h, load_library().bidiag_apply_q(h, r, trans, ncols, d_C, ldc))


def bidiag_apply_p(h, r, trans, nrows, d_C, ldc):
    _check(h, load_library().bidiag_apply_p(h, r, trans, nrows, d_C, ldc))


def bidiag_apply_q_f32(h, r, trans, ncols, d_C, ldc):
    _check(h, load_library().bidiag_apply_q_f32(h, r, trans, ncols, d_C, ldc))


def bidiag_apply_p_f32(h, r, trans, nrows, d_C, ldc):
    _check(h, load_library().bidiag_apply_p_f32(h, r, trans, nrows, d_C, ldc))


def bidiag_band_backward(h, r, d_abbar, ldab, d_Abar, ldabar, d_Arec=None, ldarec=1):
    _check(h, load_library().bidiag_band_backward(h, r, d_abbar, ldab, d_Abar, ldabar, d_Arec, ldarec))


def bidiag_band_backward_f32(h, r, d_abbar, ldab, d_Abar, ldabar, d_Arec=None, ldarec=1):
    _check(h, load_library().bidiag_band_backward_f32(h, r, d_abbar, ldab, d_Abar, ldabar, d_Arec, ldarec))


def bidiag_result_free(r):
    load_library().bidiag_result_free(r)


def bidiag_destroy(h):
    load_library().bidiag_destroy(h)


def bidiag_plan_eliminations(p, q, tree, variant, resources=1):
    lib = load_library()
    cnt = ctypes.c_int64()
    _check(None, lib.bidiag_plan_eliminations(p, q, tree, variant, resources, None, 0, ctypes.byref(cnt)))
    out = np.zeros((max(cnt.value, 1), 5), dtype=np.int32)
    _check(None, lib.bidiag_plan_eliminations(p, q, tree, variant, resources,
                                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                              cnt.value, ctypes.byref(cnt)))
    return out[:cnt.value]


def bidiag_plan_tasks(p, q, tree, variant, resources=1):
    """(tasks (ntasks x 6), levels (ntasks), critical path in Table 1 units)."""
    lib = load_library()
    cnt = ctypes.c_int64()
    cp = ctypes.c_int64()
    _check(None, lib.bidiag_plan_tasks(p, q, tree, variant, resources, None, None, 0, ctypes.byref(cnt), None))
    tasks = np.zeros((max(cnt.value, 1), 6), dtype=np.int32)
    lv = np.zeros(max(cnt.value, 1), dtype=np.int32)
    I32 = ctypes.POINTER(ctypes.c_int32)
    _check(None, lib.bidiag_plan_tasks(p, q, tree, variant, resources, tasks.ctypes.data_as(I32),
                                       lv.ctypes.data_as(I32), cnt.value, ctypes.byref(cnt), ctypes.byref(cp)))
    return tasks[:cnt.value], lv[:cnt.value], cp.value


def bidiag_plan_choose_variant(p, q, tree, resources=1):
    """(variant, critical path of BiDiag, critical path of R-BiDiag) for a p x q tile matrix."""
    v = ctypes.c_int()
    cb, cr = ctypes.c_int64(), ctypes.c_int64()
    _check(None, load_library().bidiag_plan_choose_variant(p, q, tree, resources, ctypes.byref(v), ctypes.byref(cb),
                                                          ctypes.byref(cr)))
    return v.value, cb.value, cr.value


def bidiag_plan_best_split(p, q, tree, resources=1):
    """(split, critical path) of the best three-step split for p x q tiles."""
    sp, cp = ctypes.c_int(), ctypes.c_int64()
    _check(None, load_library().bidiag_plan_best_split(p, q, tree, resources, ctypes.byref(sp), ctypes.byref(cp)))
    return sp.value, cp.value


def bidiag_plan_program(m, n, nb, ib, tree, variant, resources=1, strip_w=32):
    """Device program of a reduction: (sub-tasks (count x 8) int32, dependency array, strip width)."""
    lib = load_library()
    cnt, nd = ctypes.c_int64(), ctypes.c_int64()
    w = ctypes.c_int32()
    I32 = ctypes.POINTER(ctypes.c_int32)
    _check(None, lib.bidiag_plan_program(m, n, nb, ib, tree, variant, resources, strip_w, None, 0, ctypes.byref(cnt),
                                         None, 0, ctypes.byref(nd), ctypes.byref(w)))
    prog = np.zeros((max(cnt.value, 1), 8), dtype=np.int32)
    deps = np.zeros(max(nd.value, 1), dtype=np.int32)
    _check(None, lib.bidiag_plan_program(m, n, nb, ib, tree, variant, resources, strip_w, prog.ctypes.data_as(I32),
                                         cnt.value, ctypes.byref(cnt), deps.ctypes.data_as(I32), nd.value,
                                         ctypes.byref(nd), ctypes.byref(w)))
    return prog[:cnt.value], deps[:nd.value], w.value


def bidiag_plan_backward(m, n, nb, ib, tree, variant, resources=1, strip_w=32):
    """Adjoint program of an FP64 reduction: (sub-tasks (count x 8), forward position of each, dependency
    array, slot offsets, per-panel slot table (npanels x 4: first update slot, number of update slots,
    first panel-update slot, reduced slot or -1), column width of its update strips)."""
    lib = load_library()
    cnt, nd, ns, npi = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    wb = ctypes.c_int32()
    I32 = ctypes.POINTER(ctypes.c_int32)
    I64 = ctypes.POINTER(ctypes.c_int64)
    args = (m, n, nb, ib, tree, variant, resources, strip_w)
    _check(None, lib.bidiag_plan_backward(*args, None, None, 0, ctypes.byref(cnt), None, 0, ctypes.byref(nd), None, 0,
                                          ctypes.byref(ns), None, 0, ctypes.byref(npi), ctypes.byref(wb)))
    prog = np.zeros((max(cnt.value, 1), 8), dtype=np.int32)
    fwd = np.zeros(max(cnt.value, 1), dtype=np.int32)
    deps = np.zeros(max(nd.value, 1), dtype=np.int32)
    slot = np.zeros(max(ns.value, 1), dtype=np.int64)
    pinfo = np.zeros(max(npi.value, 1), dtype=np.int32)
    _check(None, lib.bidiag_plan_backward(*args, prog.ctypes.data_as(I32), fwd.ctypes.data_as(I32), cnt.value,
                                          ctypes.byref(cnt), deps.ctypes.data_as(I32), nd.value, ctypes.byref(nd),
                                          slot.ctypes.data_as(I64), ns.value, ctypes.byref(ns),
                                          pinfo.ctypes.data_as(I32), npi.value, ctypes.byref(npi), ctypes.byref(wb)))
    return (prog[:cnt.value], fwd[:cnt.value], deps[:nd.value], slot[:ns.value],
            pinfo[:npi.value].reshape(-1, 4), wb.value)


# ---- torch-facing wrappers ---------------------------------------------------------------------
class _CudaArray:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr, shape, strides_elems, esize=8):
        self.__cuda_array_interface__ = {
            "shape": tuple(shape), "typestr": "<f8" if esize == 8 else "<f4", "data": (int(ptr), False),
            "version": 3, "strides": tuple(esize * s for s in strides_elems)}


def _device_view(ptr, shape, strides, esize=8):
    import torch
    return torch.as_tensor(_CudaArray(ptr, shape, strides, esize), device="cuda")


def _colmajor(A):
    """Column-major FP64 / FP32 CUDA tensor (copy only if needed) and its leading dimension."""
    import torch
    if A.dtype not in (torch.float64, torch.float32) or not A.is_cuda:
        raise TypeError("A must be a float64 or float32 CUDA tensor")
    m, n = A.shape
    if A.stride(0) == 1 and (A.stride(1) >= max(1, m) or n == 1):
        return A, max(A.stride(1), m)
    Ac = A.t().contiguous().t()
    return Ac, max(m, 1)


class Handle:
    """Library handle on a CUDA device and stream (default: torch's current stream)."""

    def __init__(self, device=None, stream=None):
        import torch
        dev = torch.cuda.current_device() if device is None else int(device)
        s = torch.cuda.current_stream(dev) if stream is None else stream
        self.stream = s
        self.h = bidiag_create(dev, ctypes.c_void_p(s.cuda_stream))
        self.device = dev

    def set_option(self, option, value):
        bidiag_set_option(self.h, option, value)

    def band(self, A, nb, ib, tree="greedy", variant="bidiag"):
        tree = TREES[tree] if isinstance(tree, str) else tree
        variant = VARIANTS[variant] if isinstance(variant, str) else variant
        import torch
        Ac, lda = _colmajor(A)
        m, n = A.shape
        fn = bidiag_band_f32 if A.dtype == torch.float32 else bidiag_band
        r = fn(self.h, m, n, ctypes.c_void_p(Ac.data_ptr()), lda, nb, ib, tree, variant)
        return Result(self, r, keep=Ac)

    def band_batched(self, As, nb=None, ib=None, tree=None, variant=None):
        """Reduces a list of matrices (all float64 or all float32) in one persistent launch.

        nb / ib / tree / variant: None (autotuned or default) or a sequence with one entry per matrix
        (tree and variant entries may be names)."""
        import torch
        count = len(As)
        f32 = count > 0 and As[0].dtype == torch.float32
        cols = [_colmajor(A) for A in As]
        I64 = ctypes.c_int64 * count
        CI = ctypes.c_int * count
        m = I64(*[A.shape[0] for A in As])
        n = I64(*[A.shape[1] for A in As])
        lda = I64(*[ld for _, ld in cols])
        ptrs = (ctypes.c_void_p * count)(*[Ac.data_ptr() for Ac, _ in cols])

        def arr(v, names=None):
            if v is None:
                return None
            return CI(*[(names[x] if isinstance(x, str) else x) for x in v])

        out = (ctypes.c_void_p * count)()
        lib = load_library()
        fn = lib.bidiag_band_batched_f32 if f32 else lib.bidiag_band_batched
        _check(self.h, fn(self.h, count, m, n, ptrs, lda, arr(nb), arr(ib), arr(tree, TREES), arr(variant, VARIANTS),
                          out))
        return [Result(self, ctypes.c_void_p(out[b]), keep=cols[b][0]) for b in range(count)]

    def sync(self):
        bidiag_sync(self.h)

    def last_exec_ms(self):
        return bidiag_last_exec_ms(self.h)

    def trace(self):
        """Per-task trace of the last traced reduction: (ntasks x 4) int64 [start ns, end ns, SM, op]."""
        lib = load_library()
        cnt = ctypes.c_int64()
        _check(self.h, lib.bidiag_trace(self.h, None, 0, ctypes.byref(cnt)))
        out = np.zeros((cnt.value, 4), dtype=np.int64)
        _check(self.h, lib.bidiag_trace(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cnt.value,
                                        ctypes.byref(cnt)))
        return out

    def trace_program(self):
        """Device program of the last traced launch: (sub-tasks (count x 8) int32, dependency array)."""
        lib = load_library()
        cnt, nd = ctypes.c_int64(), ctypes.c_int64()
        _check(self.h, lib.bidiag_trace_program(self.h, None, 0, ctypes.byref(cnt), None, 0, ctypes.byref(nd)))
        prog = np.zeros((max(cnt.value, 1), 8), dtype=np.int32)
        deps = np.zeros(max(nd.value, 1), dtype=np.int32)
        I32 = ctypes.POINTER(ctypes.c_int32)
        _check(self.h, lib.bidiag_trace_program(self.h, prog.ctypes.data_as(I32), cnt.value, ctypes.byref(cnt),
                                                deps.ctypes.data_as(I32), nd.value, ctypes.byref(nd)))
        return prog[:cnt.value], deps[:nd.value]

    def close(self):
        if self.h:
            bidiag_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Result:
    """A reduction result: band B, reflector store, canonical task list."""

    def __init__(self, handle, r, keep=None):
        self.handle = handle
        self.r = r
        self._keep = keep
        lib = load_library()
        desc = Reflectors()
        _check(handle.h, lib.bidiag_result_reflectors(r, ctypes.byref(desc)))
        self.desc = desc
        self.esize = desc.elem_bytes
        ab = ctypes.c_void_p()
        ldab = ctypes.c_int64()
        n = ctypes.c_int64()
        nb = ctypes.c_int()
        getter = lib.bidiag_result_band if self.esize == 8 else lib.bidiag_result_band_f32
        _check(handle.h, getter(r, ctypes.byref(ab), ctypes.byref(ldab), ctypes.byref(n), ctypes.byref(nb)))
        self.ab_ptr, self.ldab, self.n, self.nb = ab.value, ldab.value, n.value, nb.value

    def band(self):
        """Copy of B in LAPACK upper-band storage, shape (nb + 1, n)."""
        return _device_view(self.ab_ptr, (self.nb + 1, self.n), (1, self.ldab), self.esize).clone()

    def tasks(self):
        lib = load_library()
        ptr = ctypes.POINTER(ctypes.c_int32)()
        nt = ctypes.c_int64()
        _check(self.handle.h, lib.bidiag_result_tasks(self.r, ctypes.byref(ptr), ctypes.byref(nt)))
        return np.ctypeslib.as_array(ptr, shape=(nt.value, 6)).copy()

    def tiles(self, second=False):
        """Copy of the tile buffer (grid rows x grid cols x nb x nb; [a, b] is tile (a, b), column-major)."""
        d = self.desc
        ptr = d.tiles2 if second else d.tiles
        if not ptr:
            return None
        rows = d.q if second else d.p
        cols = d.q
        nb = d.nb
        t = _device_view(ptr, (cols * rows * nb * nb,), (1,), self.esize).clone()
        return t.view(cols, rows, nb, nb).permute(1, 0, 3, 2)   # [a, b, r, c]

    def T(self):
        d = self.desc
        return _device_view(d.T, (max(d.npanels, 1), d.ib, d.nb), (d.ib * d.nb, 1, d.ib), self.esize).clone()

    def tslot(self):
        d = self.desc
        return np.ctypeslib.as_array(d.tslot, shape=(d.ntasks,)).copy()

    def apply_q(self, C, trans):
        Cc, ldc = _colmajor(C)
        fn = bidiag_apply_q if self.esize == 8 else bidiag_apply_q_f32
        fn(self.handle.h, self.r, trans, C.shape[1], ctypes.c_void_p(Cc.data_ptr()), ldc)
        if Cc.data_ptr() != C.data_ptr():
            C.copy_(Cc)
        return C

    def apply_p(self, C, trans):
        Cc, ldc = _colmajor(C)
        fn = bidiag_apply_p if self.esize == 8 else bidiag_apply_p_f32
        fn(self.handle.h, self.r, trans, C.shape[0], ctypes.c_void_p(Cc.data_ptr()), ldc)
        if Cc.data_ptr() != C.data_ptr():
            C.copy_(Cc)
        return C

    def backward(self, ab_bar, reconstruct=False):
        """dL/dA (m x n, column-major tensor) from dL/dB in band storage ((nb + 1) x n); with
        reconstruct=True also the reconstruction of A from the band and the reflectors."""
        import torch
        m = int(self.desc.m)
        dt = torch.float64 if self.esize == 8 else torch.float32
        if ab_bar.dtype != dt:
            raise TypeError("band gradient must have the result's dtype")
        Gc, ldg = _colmajor(ab_bar)
        dev = ab_bar.device
        Abar = torch.empty((self.n, m), dtype=dt, device=dev).t()
        Arec = torch.empty((self.n, m), dtype=dt, device=dev).t() if reconstruct else None
        fn = bidiag_band_backward if self.esize == 8 else bidiag_band_backward_f32
        fn(self.handle.h, self.r, ctypes.c_void_p(Gc.data_ptr()), ldg, ctypes.c_void_p(Abar.data_ptr()), max(m, 1),
           ctypes.c_void_p(Arec.data_ptr()) if reconstruct else None, max(m, 1))
        self._grad_keep = Gc     # stream-ordered use: keep the input alive until the next call
        return (Abar, Arec) if reconstruct else Abar

    def backward_workspace(self):
        """Device bytes one backward() call allocates (plans the adjoint on first use)."""
        b = ctypes.c_int64()
        _check(self.handle.h, load_library().bidiag_backward_workspace(self.handle.h, self.r, ctypes.byref(b)))
        return b.value

    def free(self):
        if self.r:
            bidiag_result_free(self.r)
            self.r = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
