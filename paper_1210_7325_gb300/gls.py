"""Python binding of the C ABI in include/gls_gb300.h (argument marshalling only).

Every step of the computation runs in the CUDA library ``libgls_gb300.so``;
this module only converts arguments.  There is no fallback: if the library is
missing or no sm_103 device is present, the calls raise.

Matrices follow the ABI's column-major convention.  A numpy array must be
Fortran-ordered; a torch tensor must have unit stride along its first axis
(e.g. the transpose ``X.t()`` of a C-contiguous (k, n) genotype tensor is the
column-major n x k matrix the ABI wants).  Host (numpy, CPU tensors, pinned or
not) and device (CUDA tensors) buffers are both accepted.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgls_gb300.so")

GLS_OK = 0
STATUS_NAMES = {
    0: "GLS_OK", 1: "GLS_ERR_INVALID_ARG", 2: "GLS_ERR_NOT_SPD", 3: "GLS_ERR_OOM",
    4: "GLS_ERR_CUDA", 5: "GLS_ERR_TIMEOUT", 6: "GLS_ERR_STATE", 7: "GLS_ERR_UNSUPPORTED",
    8: "GLS_ERR_COVARIATES_SINGULAR", 9: "GLS_ERR_IO",
}
PRECISIONS = {"fp64": 0, "bf16": 1, "fp16": 2}
GLS_FLAG_NAIVE_SPLIT = 1
GLS_FLAG_FACTOR_NATIVE = 2
GLS_FLAG_FACTOR_TENSOR = 4
GLS_FLAG_EAGER = 8
GLS_FLAG_STAGED_INPUT = 16
# the paper's algorithms for a sequence of GLS problems (gls_solve_variant)
ALGORITHMS = {"black_box": 3, "seq_gls": 4, "hp_gwas": 5, "gwfgls": 6}


class GlsError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = "", info: int = 0):
        self.status = status
        self.info = info
        name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {name}" + (f" ({detail})" if detail else "") +
                         (f" [info={info}]" if info else ""))


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("p", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("max_block_snps", ctypes.c_int64),
        ("device", ctypes.c_int32),
        ("split_terms", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("flags", ctypes.c_uint32),
        ("wait_limit_us", ctypes.c_int32),
        ("host_wait_ms", ctypes.c_int32),
        ("phenotypes", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 4),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_int64),
        ("trsm_ms", ctypes.c_double), ("trsm_launches", ctypes.c_int64),
        ("convert_ms", ctypes.c_double), ("convert_launches", ctypes.c_int64),
        ("solve_ms", ctypes.c_double), ("solve_launches", ctypes.c_int64),
        ("factor_ms", ctypes.c_double), ("factor_calls", ctypes.c_int64),
        ("h2d_ms", ctypes.c_double), ("h2d_bytes", ctypes.c_int64),
        ("h2d_copies", ctypes.c_int64),
        ("d2h_ms", ctypes.c_double), ("d2h_bytes", ctypes.c_int64),
        ("d2h_copies", ctypes.c_int64),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads (once) and returns the native library; raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"GLS CUDA library not found at {path}; build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    P = ctypes.POINTER
    lib.gls_plan_create.argtypes = [P(PlanDesc), P(vp)]
    lib.gls_plan_create.restype = i32
    lib.gls_factor.argtypes = [vp, vp, i64, vp, i64, vp, P(i64)]
    lib.gls_factor.restype = i32
    lib.gls_factor_y.argtypes = [vp, vp, i64, vp, i64, vp, i64, i32, P(i64)]
    lib.gls_factor_y.restype = i32
    lib.gls_solve_block.argtypes = [vp, vp, i64, i64, vp, i64, vp]
    lib.gls_solve_block.restype = i32
    lib.gls_solve_stream.argtypes = [vp, vp, i64, i64, vp, i64, vp]
    lib.gls_solve_stream.restype = i32
    lib.gls_solve_block_packed.argtypes = [vp, vp, i64, i64, vp, i64, vp]
    lib.gls_solve_block_packed.restype = i32
    lib.gls_solve_stream_packed.argtypes = [vp, vp, i64, i64, vp, i64, vp]
    lib.gls_solve_stream_packed.restype = i32
    lib.gls_solve_file.argtypes = [vp, ctypes.c_char_p, i64, i32, i64, i64, vp, i64, vp]
    lib.gls_solve_file.restype = i32
    lib.gls_synchronize.argtypes = [vp]
    lib.gls_synchronize.restype = i32
    lib.gls_plan_stream.argtypes = [vp]
    lib.gls_plan_stream.restype = vp
    lib.gls_plan_wait_event.argtypes = [vp, vp]
    lib.gls_plan_wait_event.restype = i32
    lib.gls_plan_operand_precision.argtypes = [vp]
    lib.gls_plan_operand_precision.restype = i32
    lib.gls_destroy.argtypes = [vp]
    lib.gls_destroy.restype = i32
    lib.gls_plan_footprint_bytes.argtypes = [P(PlanDesc)]
    lib.gls_plan_footprint_bytes.restype = ctypes.c_size_t
    lib.gls_status_string.argtypes = [i32]
    lib.gls_status_string.restype = ctypes.c_char_p
    lib.gls_last_error.argtypes = []
    lib.gls_last_error.restype = ctypes.c_char_p
    lib.gls_version.argtypes = []
    lib.gls_version.restype = i32
    lib.gls_batch_create.argtypes = [P(vp), i32, P(vp)]
    lib.gls_batch_create.restype = i32
    lib.gls_batch_solve.argtypes = [vp, P(vp), P(i64), P(i64), P(vp), P(i64), P(vp), i32]
    lib.gls_batch_solve.restype = i32
    lib.gls_batch_destroy.argtypes = [vp]
    lib.gls_batch_destroy.restype = i32
    lib.gls_plan_set_timing.argtypes = [vp, i32]
    lib.gls_plan_set_timing.restype = i32
    lib.gls_plan_stats.argtypes = [vp, P(Stats)]
    lib.gls_plan_stats.restype = i32
    lib.gls_plan_get_factor.argtypes = [vp, vp, i64, vp, i64]
    lib.gls_plan_get_factor.restype = i32
    lib.gls_solve_variant.argtypes = [vp, i32, vp, i64, vp, i64, vp, vp, i64, i64, vp, i64, vp]
    lib.gls_solve_variant.restype = i32
    _lib = lib
    return lib


def last_error() -> str:
    return load().gls_last_error().decode()


def _check(status: int, where: str, info: int = 0):
    if status != GLS_OK:
        raise GlsError(status, where, last_error(), info)


def make_desc(n, p, max_block_snps, precision="fp64", device=0, stream=None, split_terms=0,
              flags=0, wait_limit_us=0, host_wait_ms=0, phenotypes=1) -> PlanDesc:
    d = PlanDesc()
    d.n = int(n)
    d.p = int(p)
    d.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    d.max_block_snps = int(max_block_snps)
    d.device = int(device)
    d.split_terms = int(split_terms)
    d.stream = stream
    d.flags = int(flags)
    d.wait_limit_us = int(wait_limit_us)
    d.host_wait_ms = int(host_wait_ms)
    d.phenotypes = int(phenotypes)
    return d


def footprint_bytes(n, p, max_block_snps, precision="fp64", split_terms=0, flags=0,
                    phenotypes=1) -> int:
    return int(load().gls_plan_footprint_bytes(
        ctypes.byref(make_desc(n, p, max_block_snps, precision, split_terms=split_terms,
                               flags=flags, phenotypes=phenotypes))))


# ------------------------------------------------------------------ marshalling
def _colmajor(a, rows: int, itemsize: int, name: str):
    """(pointer, leading dimension in elements) of a column-major matrix."""
    if a is None:
        return None, max(rows, 1)
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.element_size() != itemsize:
                raise TypeError(f"{name}: element size {a.element_size()} != {itemsize}")
            if a.dim() == 1:
                return ctypes.c_void_p(a.data_ptr()), max(rows, 1)
            if a.dim() != 2 or (a.shape[1] > 1 and a.stride(0) != 1):
                raise ValueError(f"{name}: torch tensor must be column-major (stride(0) == 1)")
            ld = a.stride(1) if a.shape[1] > 1 else max(a.shape[0], 1)
            return ctypes.c_void_p(a.data_ptr()), ld
    except ImportError:
        pass
    import numpy as np
    if not isinstance(a, np.ndarray):
        raise TypeError(f"{name}: expected a numpy array or torch tensor")
    if a.itemsize != itemsize:
        raise TypeError(f"{name}: element size {a.itemsize} != {itemsize}")
    if a.ndim == 1:
        if not a.flags.c_contiguous:
            raise ValueError(f"{name}: vector must be contiguous")
        return ctypes.c_void_p(a.ctypes.data), max(rows, 1)
    if a.ndim != 2 or not a.flags.f_contiguous:
        raise ValueError(f"{name}: numpy matrix must be Fortran-ordered (column-major)")
    return ctypes.c_void_p(a.ctypes.data), max(a.shape[0], 1)


def packed_rows(n: int) -> int:
    """Bytes per SNP column of the 2-bit packed genotype layout."""
    return (int(n) + 3) // 4


def pack_genotypes(X, allow_code3=False):
    """Packs n x k genotype codes 0..2 (int8 or uint8, numpy or torch) four to a
    byte: column j -> ceil(n/4) bytes, genotype i in bits 2 (i mod 4) ..
    2 (i mod 4) + 1 of byte i // 4 (the layout of gls_solve_*_packed).  The
    result is column-major uint8 in the same library (and device) as X.  Works
    on byte views: the temporaries are about n x k / 4 bytes each.
    The library reads code 3 as the value 3; it is refused here unless
    allow_code3, because 2-bit genotype files of other tools give the codes
    other meanings (one of them often marks a missing call)."""
    top = 3 if allow_code3 else 2
    n = X.shape[0]
    k = X.shape[1] if X.ndim == 2 else 1
    nb = packed_rows(n)
    try:
        import torch
        if isinstance(X, torch.Tensor):
            if X.dtype not in (torch.int8, torch.uint8):
                raise TypeError("packed genotype codes must be int8 or uint8")
            x = X.reshape(n, k)
            if x.numel() and (int(x.min()) < 0 or int(x.max()) > top):
                raise ValueError(f"packed genotype codes must be in 0..{top}")
            x = x.view(torch.uint8)  # same bits for 0..3
            if n % 4:
                pad = torch.zeros((4 * nb, k), dtype=torch.uint8, device=X.device)
                pad[:n] = x
                x = pad
            q = x.reshape(nb, 4, k)
            b = q[:, 0] | (q[:, 1] << 2) | (q[:, 2] << 4) | (q[:, 3] << 6)
            out = torch.empty((k, nb), dtype=torch.uint8, device=X.device).t()
            out.copy_(b)
            return out
    except ImportError:
        pass
    import numpy as np
    x = np.asarray(X)
    if x.dtype not in (np.int8, np.uint8):
        raise TypeError("packed genotype codes must be int8 or uint8")
    x = x.reshape(n, k, order="F")
    if x.size and (int(x.min()) < 0 or int(x.max()) > top):
        raise ValueError(f"packed genotype codes must be in 0..{top}")
    x = x.view(np.uint8)
    pad = np.zeros((4 * nb, k), dtype=np.uint8)  # row-major: row 4 b + q -> q[b, q]
    pad[:n] = x
    q = pad.reshape(nb, 4, k)
    b = q[:, 0] | (q[:, 1] << 2) | (q[:, 2] << 4) | (q[:, 3] << 6)
    return np.asfortranarray(b.astype(np.uint8))


def _ptr(a):
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return ctypes.c_void_p(a.data_ptr())
    except ImportError:
        pass
    return ctypes.c_void_p(a.ctypes.data)


class Plan:
    """One GLS sequence: ``factor`` (setup of Alg. 5) then ``solve_block`` /
    ``solve_stream`` over SNP blocks.  Thin wrapper over the C ABI."""

    def __init__(self, n, p, max_block_snps, precision="fp64", device=0, stream=None,
                 split_terms=0, flags=0, wait_limit_us=0, host_wait_ms=0, phenotypes=1):
        lib = load()
        self.n, self.p, self.kmax = int(n), int(p), int(max_block_snps)
        self.precision = precision
        self.phenotypes = int(phenotypes)  # capacity t of the plan
        self.t = 1                         # phenotypes of the last factor
        self._desc = make_desc(n, p, max_block_snps, precision, device, stream, split_terms,
                               flags, wait_limit_us, host_wait_ms, phenotypes)
        h = ctypes.c_void_p()
        _check(lib.gls_plan_create(ctypes.byref(self._desc), ctypes.byref(h)), "gls_plan_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def operand_precision(self) -> str:
        """The precision the plan's tensor-core operands use ("bf16", "fp16";
        "fp64" for the binary64 path): a BF16 plan with n < 2048 uses FP16."""
        code = load().gls_plan_operand_precision(self._h)
        return {v: k for k, v in PRECISIONS.items()}[code]

    @property
    def stream(self) -> int:
        return int(load().gls_plan_stream(self._h) or 0)

    def wait_event(self, event):
        """Orders the plan's later work after ``event`` (a ``torch.cuda.Event``
        recorded on the stream that produced the next calls' device inputs, or
        a raw cudaEvent_t handle)."""
        h = getattr(event, "cuda_event", event)
        _check(load().gls_plan_wait_event(self._h, ctypes.c_void_p(int(h))),
               "gls_plan_wait_event")

    def factor(self, M, XL, y):
        """M: n x n column-major (lower triangle read) or None to keep the previous
        factor; XL: n x (p-1) column-major or None; y: an n vector, or an n x t
        column-major matrix of t <= phenotypes phenotypes (gls_factor_y; then B
        holds p x t values per SNP, column i t + j)."""
        lib = load()
        pm, ldm = _colmajor(M, self.n, 8, "M")
        px, ldx = _colmajor(XL, self.n, 8, "XL")
        t = 1 if (y.ndim == 1 or y.shape[1] == 1) else int(y.shape[1])
        py, ldy = _colmajor(y, self.n, 8, "y")
        info = ctypes.c_int64(0)
        st = lib.gls_factor_y(self._h, pm, ldm, px, ldx, py, ldy, t, ctypes.byref(info))
        _check(st, "gls_factor_y", info.value)
        self.t = t

    def solve_block(self, XR, B, status=None, k=None):
        """XR: n x k int8 column-major; B: p x k float64 column-major (output);
        status: k int32 or None."""
        lib = load()
        px, ldx = _colmajor(XR, self.n, 1, "XR")
        pb, ldb = _colmajor(B, self.p, 8, "B")
        if k is None:
            k = XR.shape[1] if XR.ndim == 2 else 1
        _check(lib.gls_solve_block(self._h, px, ldx, int(k), pb, ldb, _ptr(status)),
               "gls_solve_block")

    def solve_stream(self, XR, B, status=None, m=None):
        lib = load()
        px, ldx = _colmajor(XR, self.n, 1, "XR")
        pb, ldb = _colmajor(B, self.p, 8, "B")
        if m is None:
            m = XR.shape[1]
        _check(lib.gls_solve_stream(self._h, px, ldx, int(m), pb, ldb, _ptr(status)),
               "gls_solve_stream")

    def solve_file(self, path, m, B, status=None, offset=0, packed=False, ldx=None):
        """The SNP stream read from a file (gls_solve_file): m columns of int8
        codes (or the 2-bit packed layout) from byte `offset`, ldx bytes apart
        (default n, or ceil(n/4) packed)."""
        lib = load()
        if ldx is None:
            ldx = packed_rows(self.n) if packed else self.n
        pb, ldb = _colmajor(B, self.p, 8, "B")
        _check(lib.gls_solve_file(self._h, os.fsencode(path), int(offset), int(bool(packed)),
                                  int(ldx), int(m), pb, ldb, _ptr(status)), "gls_solve_file")

    def solve_block_packed(self, XP, B, status=None, k=None):
        """XP: ceil(n/4) x k uint8 column-major, 2-bit codes (see pack_genotypes)."""
        lib = load()
        px, ldx = _colmajor(XP, packed_rows(self.n), 1, "XP")
        pb, ldb = _colmajor(B, self.p, 8, "B")
        if k is None:
            k = XP.shape[1] if XP.ndim == 2 else 1
        _check(lib.gls_solve_block_packed(self._h, px, ldx, int(k), pb, ldb, _ptr(status)),
               "gls_solve_block_packed")

    def solve_stream_packed(self, XP, B, status=None, m=None):
        lib = load()
        px, ldx = _colmajor(XP, packed_rows(self.n), 1, "XP")
        pb, ldb = _colmajor(B, self.p, 8, "B")
        if m is None:
            m = XP.shape[1]
        _check(lib.gls_solve_stream_packed(self._h, px, ldx, int(m), pb, ldb, _ptr(status)),
               "gls_solve_stream_packed")

    def solve_variant(self, algorithm, M, XL, y, XR, B, status=None, k=None):
        """One of the paper's algorithms ("black_box" Alg. 3, "seq_gls" Alg. 4,
        "hp_gwas" Alg. 5, "gwfgls" Alg. 6) on device buffers: b_i of the k
        SNP columns of XR into B (p x k).  The comparison algorithms leave the
        plan without a factor; "hp_gwas" leaves its factor in place."""
        lib = load()
        alg = ALGORITHMS[algorithm] if isinstance(algorithm, str) else int(algorithm)
        pm, ldm = _colmajor(M, self.n, 8, "M")
        pl_, ldl = _colmajor(XL, self.n, 8, "XL")
        py, _ = _colmajor(y, self.n, 8, "y")
        px, ldx = _colmajor(XR, self.n, 1, "XR")
        pb, ldb = _colmajor(B, self.p, 8, "B")
        if k is None:
            k = XR.shape[1] if XR.ndim == 2 else 1
        _check(lib.gls_solve_variant(self._h, alg, pm, ldm, pl_, ldl, py, px, ldx, int(k), pb,
                                     ldb, _ptr(status)), "gls_solve_variant")

    def get_factor(self, L=None, Zinv=None):
        """Copies L and L^{-1} (n x n column-major, host or device) of the last factor."""
        pl, ldl = _colmajor(L, self.n, 8, "L")
        pz, ldz = _colmajor(Zinv, self.n, 8, "Zinv")
        _check(load().gls_plan_get_factor(self._h, pl, ldl, pz, ldz), "gls_plan_get_factor")

    def set_timing(self, enable: bool = True):
        """Enables per-kernel device timing (and resets the counters)."""
        _check(load().gls_plan_set_timing(self._h, int(bool(enable))), "gls_plan_set_timing")

    def stats(self) -> dict:
        st = Stats()
        _check(load().gls_plan_stats(self._h, ctypes.byref(st)), "gls_plan_stats")
        return st.as_dict()

    def synchronize(self):
        _check(load().gls_synchronize(self._h), "gls_synchronize")

    def close(self):
        if getattr(self, "_h", None):
            load().gls_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several factored mixed-precision plans solved by one persistent launch
    (gls_batch_create / gls_batch_solve).  Device buffers only."""

    def __init__(self, plans):
        lib = load()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(lib.gls_batch_create(arr, len(self.plans), ctypes.byref(h)), "gls_batch_create")
        self._h = h

    def solve(self, XRs, Bs, statuses=None, ks=None, group=0):
        """XRs[i]: n_i x k_i int8 column-major device tensors (e.g. X.t() of a
        (k_i, n_i) tensor); Bs[i]: p_i x k_i float64 column-major device tensors."""
        lib = load()
        n = len(self.plans)
        xs, lx, bs, lb = [], [], [], []
        for pl, X, B in zip(self.plans, XRs, Bs):
            px, ldx = _colmajor(X, pl.n, 1, "XR")
            pb, ldb = _colmajor(B, pl.p, 8, "B")
            xs.append(px.value or 0)
            lx.append(ldx)
            bs.append(pb.value or 0)
            lb.append(ldb)
        if ks is None:
            ks = [X.shape[1] for X in XRs]
        VP, I64 = ctypes.c_void_p * n, ctypes.c_int64 * n
        st = None
        if statuses is not None:
            st = VP(*[(_ptr(s).value if s is not None else None) for s in statuses])
        _check(lib.gls_batch_solve(self._h, VP(*xs), I64(*lx), I64(*[int(k) for k in ks]),
                                   VP(*bs), I64(*lb), st, int(group)), "gls_batch_solve")

    def close(self):
        if getattr(self, "_h", None):
            load().gls_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
