"""Python binding of libepi (ctypes).

Marshalling only: every step of a search runs in the library's CUDA kernels.
PyTorch provides the CUDA stream (and, for device-resident inputs, the device
memory); numpy arrays are host buffers.  There is no fallback: if the shared
library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import re
import threading
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libepi.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "epi.h")

EPI_OK, EPI_EINVAL, EPI_ENOMEM, EPI_ECUDA, EPI_EUNSUPPORTED, EPI_ETIMEOUT, EPI_EOVERFLOW = range(7)
PATHS = {"auto": 0, "popc": 1, "tc": 2}
TC_VARIANTS = {"auto": 0, "separate": 1}
MAX_ORDER = 8

RESULT_DTYPE = np.dtype([("snp", "<u4", (MAX_ORDER,)), ("mi", "<f8"), ("mi_f32", "<f4"),
                         ("order", "<u4"), ("rank", "<u8")])
assert RESULT_DTYPE.itemsize == 56


class EpiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libepi status {status}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None
_live_datasets: "weakref.WeakSet" = weakref.WeakSet()
_live_contexts: "weakref.WeakSet" = weakref.WeakSet()


@atexit.register
def _close_all():
    # datasets before their contexts, while the CUDA runtime is still up
    for ds in list(_live_datasets):
        try:
            ds.close()
        except Exception:
            pass
    for ctx in list(_live_contexts):
        try:
            ctx.close()
        except Exception:
            pass


def exported_names() -> list[str]:
    """Function names declared in include/epi.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(epi_[a-z0-9_]+)\s*\(",
                                 text, flags=re.M)))


class ProposerOpts(C.Structure):
    _fields_ = [("top_triples", C.c_int), ("budget", C.c_int), ("top_n", C.c_int), ("chunk", C.c_int64),
                ("quad_features", C.c_int)]


class ProposerStats(C.Structure):
    _fields_ = [("candidates", C.c_uint64), ("kept", C.c_uint64), ("proposals", C.c_uint64),
                ("ms_lower", C.c_double), ("ms_rank", C.c_double), ("ms_rescore", C.c_double),
                ("exact_in_proposals", C.c_int32)]


class TrainOpts(C.Structure):
    _fields_ = [("top_triples", C.c_int), ("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_float),
                ("wd", C.c_float), ("tail_fraction", C.c_float), ("seed", C.c_uint64), ("target", C.c_int)]


def load(path: str | None = None):
    """Load libepi (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise OSError(f"libepi is not built ({p} missing); run paper_2201_02460_gb300.build.build()")
        lib = C.CDLL(p)
        V, P = C.c_void_p, C.c_void_p
        i32, i64, u64 = C.c_int, C.c_int64, C.c_uint64
        lib.epi_last_error.restype = C.c_char_p
        lib.epi_last_error.argtypes = []
        lib.epi_create.restype = i32
        lib.epi_create.argtypes = [i32, V, C.POINTER(V)]
        lib.epi_destroy.restype = None
        lib.epi_destroy.argtypes = [V]
        lib.epi_dataset_create.restype = i32
        lib.epi_dataset_create.argtypes = [V, P, P, i64, i64, i32, C.POINTER(V)]
        lib.epi_dataset_destroy.restype = None
        lib.epi_dataset_destroy.argtypes = [V]
        lib.epi_dataset_info.restype = i32
        lib.epi_dataset_info.argtypes = [V, P, P, P, P]
        lib.epi_search.restype = i32
        lib.epi_search.argtypes = [V, i32, i32, i32, P, P, P]
        lib.epi_search_range.restype = i32
        lib.epi_search_range.argtypes = [V, i32, i32, i32, u64, u64, P, P, P]
        lib.epi_search_async.restype = i32
        lib.epi_search_async.argtypes = [V, i32, i32, i32, P, P, P, P]
        lib.epi_tables.restype = i32
        lib.epi_tables.argtypes = [V, i32, P, i64, P]
        lib.epi_score_tables.restype = i32
        lib.epi_score_tables.argtypes = [V, i32, P, i64, P, P]
        lib.epi_kernel_launches.restype = u64
        lib.epi_kernel_launches.argtypes = [V]
        lib.epi_score_all.restype = i32
        lib.epi_score_all.argtypes = [V, i32, P]
        lib.epi_unrank.restype = i32
        lib.epi_unrank.argtypes = [V, i32, P, i64, P]
        lib.epi_features5.restype = i32
        lib.epi_features5.argtypes = [V, P, P, P, P, P, i64, P]
        lib.epi_candidates5.restype = i32
        lib.epi_candidates5.argtypes = [V, P, i64, i64, i64, P, P, P]
        lib.epi_lookup.restype = i32
        lib.epi_lookup.argtypes = [V, i32, P, P, i64, P]
        lib.epi_topk.restype = i32
        lib.epi_topk.argtypes = [V, P, P, i64, i32, P, P, P]
        lib.epi_search_threshold.restype = i32
        lib.epi_search_threshold.argtypes = [V, C.c_int, C.c_double, i64, P, i64, P, C.POINTER(C.c_int64)]
        lib.epi_score5.restype = i32
        lib.epi_score5.argtypes = [V, P, i64, P]
        lib.epi_heuristic5.restype = i32
        lib.epi_heuristic5.argtypes = [V, P, i64, C.c_int, P]
        lib.epi_mlp_create.restype = i32
        lib.epi_mlp_create.argtypes = [V, i32, i32, u64, C.POINTER(V)]
        lib.epi_mlp_destroy.restype = None
        lib.epi_mlp_destroy.argtypes = [V]
        lib.epi_mlp_num_params.restype = i64
        lib.epi_mlp_num_params.argtypes = [V]
        lib.epi_mlp_get_params.restype = i32
        lib.epi_mlp_get_params.argtypes = [V, P]
        lib.epi_mlp_set_params.restype = i32
        lib.epi_mlp_set_params.argtypes = [V, P]
        lib.epi_mlp_forward.restype = i32
        lib.epi_mlp_forward.argtypes = [V, P, i64, P]
        lib.epi_mlp_gradients.restype = i32
        lib.epi_mlp_gradients.argtypes = [V, P, P, i64, P, P]
        lib.epi_mlp_train_step.restype = i32
        lib.epi_mlp_train_step.argtypes = [V, P, P, i64, C.c_float, C.c_float, P]
        lib.epi_mlp_set_forward_path.restype = i32
        lib.epi_mlp_set_forward_path.argtypes = [V, i32]
        lib.epi_mlp_num_inputs.restype = i32
        lib.epi_mlp_num_inputs.argtypes = [V]
        lib.epi_mlp_set_input_norm.restype = i32
        lib.epi_mlp_set_input_norm.argtypes = [V, P, P]
        lib.epi_mlp_get_input_norm.restype = i32
        lib.epi_mlp_get_input_norm.argtypes = [V, P, P]
        lib.epi_proposer_search.restype = i32
        lib.epi_proposer_search.argtypes = [V, V, C.POINTER(ProposerOpts), P, P, P, C.POINTER(ProposerStats)]
        lib.epi_proposer_train.restype = i32
        lib.epi_proposer_train.argtypes = [V, P, i32, C.POINTER(TrainOpts), P]
        lib.epi_autotune.restype = i32
        lib.epi_autotune.argtypes = [V, i32, P]
        lib.epi_tune_save.restype = i32
        lib.epi_tune_save.argtypes = [V, C.c_char_p]
        lib.epi_tune_load.restype = i32
        lib.epi_tune_load.argtypes = [V, C.c_char_p]
        lib.epi_search_batched.restype = i32
        lib.epi_search_batched.argtypes = [V, P, P, P, i32, i32, P, P, P]
        lib.epi_debug_counts.restype = i32
        lib.epi_debug_counts.argtypes = [V, i32, P]
        lib.epi_profile_begin.restype = i32
        lib.epi_profile_begin.argtypes = [V]
        lib.epi_profile_end.restype = i32
        lib.epi_profile_end.argtypes = [V, P, P]
        lib.epi_profile_waits.restype = i32
        lib.epi_profile_waits.argtypes = [V, P]
        lib.epi_tc_rate.restype = i32
        lib.epi_tc_rate.argtypes = [V, i32, i64, P]
        lib.epi_count_variant.restype = i32
        lib.epi_count_variant.argtypes = [V, i32, i32, P, P, P]
        lib.epi_set_wait_limit.restype = i32
        lib.epi_set_wait_limit.argtypes = [V, u64]
        lib.epi_inject_alloc_failure.restype = i32
        lib.epi_inject_alloc_failure.argtypes = [V, i64]
        lib.epi_set_tc_variant.restype = i32
        lib.epi_set_tc_variant.argtypes = [V, i32]
        if path is None:
            _lib = lib
        return lib


def _check(rc: int):
    if rc != EPI_OK:
        raise EpiError(rc, load().epi_last_error().decode(errors="replace"))


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _current_stream_handle():
    import torch
    return torch.cuda.current_stream().cuda_stream


class Context:
    """A libepi context on one CUDA device and stream (torch's current stream
    by default)."""

    def __init__(self, device: int = 0, stream=None):
        lib = load()
        if stream is None:
            import torch
            with torch.cuda.device(device):
                stream = torch.cuda.current_stream().cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.device = device
        self.stream = stream
        h = C.c_void_p()
        _check(lib.epi_create(device, C.c_void_p(stream), C.byref(h)))
        self._h = h
        _live_contexts.add(self)

    @property
    def handle(self):
        return self._h

    def kernel_launches(self) -> int:
        return int(load().epi_kernel_launches(self._h))

    def profile_begin(self):
        _check(load().epi_profile_begin(self._h))

    def profile_end(self) -> tuple[float, int]:
        """(summed milliseconds, launches) of the counting kernel since
        profile_begin."""
        ms = C.c_double(0.0)
        n = C.c_int64(0)
        _check(load().epi_profile_end(self._h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def profile_waits(self) -> dict:
        """Per-role wait cycles of the last profiled tensor-core search."""
        out = np.zeros(8, dtype=np.float64)
        _check(load().epi_profile_waits(self._h, _np_ptr(out)))
        names = ["mma_wait_a", "mma_wait_b", "mma_wait_acc", "prod_wait_stage", "prod_wait_acc", "epi_wait_acc",
                 "tma_wait_stage", "mma_loop"]
        return {k: float(v) for k, v in zip(names, out)}

    def set_wait_limit(self, ns: int):
        """Limit of the tensor-core kernel's pipeline waits (0: default)."""
        _check(load().epi_set_wait_limit(self._h, int(ns)))

    def inject_alloc_failure(self, after: int):
        """Make the device allocation after `after` further ones fail once
        (negative: cancel)."""
        _check(load().epi_inject_alloc_failure(self._h, int(after)))

    def set_tc_variant(self, variant: str):
        """Tensor-core counting variant: "auto" (combined classes where they
        fit) or "separate"."""
        _check(load().epi_set_tc_variant(self._h, TC_VARIANTS[variant]))

    def tc_rate(self, stages: int = 1 << 19, shape: int = 0) -> dict:
        """Rate of the tensor pipe for a counting-path MMA (shape 0: E4M3
        M128 N128 K32; shape 1: E5M2 M128 N256 K32), measured with one CTA
        per SM issuing it back to back."""
        out = np.zeros(4, dtype=np.float64)
        _check(load().epi_tc_rate(self._h, int(shape), int(stages), _np_ptr(out)))
        return dict(tflops=float(out[0]), mac_per_clk_sm=float(out[1]), ms=float(out[2]), sm_mhz=float(out[3]))

    def close(self):
        if getattr(self, "_h", None):
            load().epi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Dataset:
    """Genotype tables of one dataset on the context's device.

    geno [n_snps, n_samples] uint8 in {0,1,2}, pheno [n_samples] uint8 in
    {0,1}; numpy arrays (host) or torch CUDA tensors (device)."""

    def __init__(self, ctx: Context, geno, pheno):
        lib = load()
        self.ctx = ctx
        on_dev = hasattr(geno, "is_cuda") and geno.is_cuda
        if on_dev:
            import torch
            if geno.dtype != torch.uint8 or pheno.dtype != torch.uint8:
                raise TypeError("device inputs must be torch.uint8")
            geno = geno.contiguous()
            pheno = pheno.contiguous()
            n, m = geno.shape
            gp, pp = C.c_void_p(geno.data_ptr()), C.c_void_p(pheno.data_ptr())
            keep = (geno, pheno)
        else:
            geno = np.ascontiguousarray(geno, dtype=np.uint8)
            pheno = np.ascontiguousarray(pheno, dtype=np.uint8)
            n, m = geno.shape
            gp, pp = _np_ptr(geno), _np_ptr(pheno)
            keep = (geno, pheno)
        if pheno.shape[0] != m:
            raise ValueError("pheno length must equal the number of samples")
        h = C.c_void_p()
        _check(lib.epi_dataset_create(ctx.handle, gp, pp, n, m, 1 if on_dev else 0, C.byref(h)))
        del keep
        self._h = h
        _live_datasets.add(self)
        info = np.zeros(4, dtype=np.int64)
        _check(lib.epi_dataset_info(h, _np_ptr(info[0:]), _np_ptr(info[1:]), _np_ptr(info[2:]), _np_ptr(info[3:])))
        self.n_snps, self.n_samples, self.n_cases, self.n_controls = (int(x) for x in info)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().epi_dataset_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SearchResult:
    def __init__(self, recs: np.ndarray, counts: np.ndarray | None, order: int):
        self.records = recs
        self.order = order
        self.combs = recs["snp"][:, :order].astype(np.int64)
        self.mi = recs["mi"].copy()
        self.mi_f32 = recs["mi_f32"].copy()
        self.rank = recs["rank"].copy()
        self.counts = counts

    def __len__(self):
        return len(self.records)


def search(ds: Dataset, order: int, top_n: int, path: str = "auto", rank_range=None,
           with_counts: bool = True) -> SearchResult:
    lib = load()
    out = np.zeros(top_n, dtype=RESULT_DTYPE)
    counts = np.zeros((top_n, 2, 3 ** order), dtype=np.uint32) if with_counts else None
    n_out = C.c_int(0)
    cp = _np_ptr(counts) if with_counts else None
    if rank_range is None:
        _check(lib.epi_search(ds.handle, order, top_n, PATHS[path], _np_ptr(out), cp, C.byref(n_out)))
    else:
        r0, r1 = rank_range
        _check(lib.epi_search_range(ds.handle, order, top_n, PATHS[path], int(r0), int(min(r1, 2 ** 64 - 1)),
                                    _np_ptr(out), cp, C.byref(n_out)))
    n = n_out.value
    return SearchResult(out[:n], counts[:n] if with_counts else None, order)


def search_async(ds: Dataset, order: int, top_n: int, out_dev, counts_dev, n_out_dev, status_dev,
                 path: str = "auto"):
    """Device-side search into torch CUDA tensors (out_dev: uint8 [top_n*56],
    counts_dev: int32 [top_n, 2, 3^k] or None, n_out_dev / status_dev: int32 [1])."""
    lib = load()
    cp = C.c_void_p(counts_dev.data_ptr()) if counts_dev is not None else None
    _check(lib.epi_search_async(ds.handle, order, top_n, PATHS[path], C.c_void_p(out_dev.data_ptr()), cp,
                                C.c_void_p(n_out_dev.data_ptr()), C.c_void_p(status_dev.data_ptr())))


def autotune(ds: Dataset, order: int) -> dict:
    """Time the launch shapes and paths for this dataset's size bucket and
    keep the fastest in the context (see epi_autotune)."""
    out = np.zeros(4, dtype=np.int32)
    _check(load().epi_autotune(ds.handle, order, _np_ptr(out)))
    return dict(row_group=int(out[0]), tile=int(out[1]), slots=int(out[2]),
                path={1: "popc", 2: "tc"}.get(int(out[3]), "?"))


def tune_save(ctx: Context, path: str):
    _check(load().epi_tune_save(ctx.handle, path.encode()))


def tune_load(ctx: Context, path: str):
    _check(load().epi_tune_load(ctx.handle, path.encode()))


def search_batched(ctx: Context, datasets, orders, top_ns, path: str = "auto",
                   with_counts: bool = True) -> list:
    """One batched search over several datasets (see epi_search_batched);
    returns one SearchResult per dataset."""
    lib = load()
    n = len(datasets)
    orders = [int(x) for x in orders]
    top_ns = [int(x) for x in top_ns]
    outs = [np.zeros(t, dtype=RESULT_DTYPE) for t in top_ns]
    cnts = [np.zeros((t, 2, 3 ** k), dtype=np.uint32) for t, k in zip(top_ns, orders)] if with_counts else None
    h = (C.c_void_p * n)(*[d.handle.value for d in datasets])
    o_arr = (C.c_int * n)(*orders)
    t_arr = (C.c_int * n)(*top_ns)
    out_p = (C.c_void_p * n)(*[o.ctypes.data for o in outs])
    cnt_p = (C.c_void_p * n)(*[c.ctypes.data for c in cnts]) if with_counts else None
    n_out = (C.c_int * n)()
    _check(lib.epi_search_batched(ctx.handle, h, o_arr, t_arr, n, PATHS[path], out_p, cnt_p, n_out))
    return [SearchResult(outs[i][: n_out[i]], cnts[i][: n_out[i]] if with_counts else None, orders[i])
            for i in range(n)]


def debug_counts(ds: Dataset, order: int) -> np.ndarray:
    """Every combination's table as the tensor-core path counts it,
    [C(n,k), 2, 3^k] in lexicographic rank order (small datasets only)."""
    import math
    lib = load()
    total = math.comb(ds.n_snps, order)
    out = np.zeros((total, 2, 3 ** order), dtype=np.uint32)
    _check(lib.epi_debug_counts(ds.handle, order, _np_ptr(out)))
    return out


COUNT_VARIANTS = {"popc": 0, "lut": 1, "mma_b1": 2}


def count_variant(ds: Dataset, order: int, variant: str, with_tables: bool = False) -> dict:
    """Every order-`order` table counted with one last-level instruction
    (epi_count_variant): checksum, kernel milliseconds and, optionally, the
    tables [C(n,k), 2, 3^k] in rank order."""
    import math
    lib = load()
    tabs = np.zeros((math.comb(ds.n_snps, order), 2, 3 ** order), dtype=np.uint32) if with_tables else None
    cs = C.c_uint64(0)
    ms = C.c_double(0.0)
    _check(lib.epi_count_variant(ds.handle, order, COUNT_VARIANTS[variant],
                                 _np_ptr(tabs) if tabs is not None else None, C.byref(cs), C.byref(ms)))
    return dict(checksum=int(cs.value), ms=float(ms.value), tables=tabs)


def tables(ds: Dataset, combs) -> np.ndarray:
    lib = load()
    combs = np.ascontiguousarray(combs, dtype=np.uint32)
    if combs.ndim != 2:
        raise ValueError("combs must be [count, order]")
    count, order = combs.shape
    out = np.zeros((count, 2, 3 ** order), dtype=np.uint32)
    _check(lib.epi_tables(ds.handle, order, _np_ptr(combs), count, _np_ptr(out)))
    return out


def score_tables(ds: Dataset, order: int, tabs) -> tuple[np.ndarray, np.ndarray]:
    lib = load()
    tabs = np.ascontiguousarray(tabs, dtype=np.uint32)
    count = tabs.shape[0]
    f32 = np.zeros(count, dtype=np.float32)
    f64 = np.zeros(count, dtype=np.float64)
    _check(lib.epi_score_tables(ds.handle, order, _np_ptr(tabs), count, _np_ptr(f32), _np_ptr(f64)))
    return f32, f64


# ---------------------------------------------------------------------------
# learned proposer (device buffers are torch CUDA tensors)
# ---------------------------------------------------------------------------

def _dptr(t):
    return C.c_void_p(t.data_ptr())


def search_threshold(ds: Dataset, order: int, threshold: float, capacity: int, chunk: int = 0,
                     with_counts: bool = True) -> tuple[SearchResult, int]:
    """Every combination with MI >= threshold, best first (at most
    `capacity` returned), and how many qualify (epi_search_threshold)."""
    out = np.zeros(max(capacity, 1), dtype=RESULT_DTYPE)
    counts = np.zeros((max(capacity, 1), 2, 3 ** order), dtype=np.uint32) if with_counts else None
    n = C.c_int64(0)
    _check(load().epi_search_threshold(ds.handle, order, float(threshold), chunk, _np_ptr(out), capacity,
                                       _np_ptr(counts) if with_counts else None, C.byref(n)))
    m = min(capacity, n.value)
    return SearchResult(out[:m], counts[:m] if with_counts else None, order), n.value


def score_all(ds: Dataset, order: int):
    """Every combination's FP32 MI by lexicographic rank (torch float32 on
    the dataset's device)."""
    import math
    import torch
    out = torch.empty(math.comb(ds.n_snps, order), dtype=torch.float32, device=f"cuda:{ds.ctx.device}")
    _check(load().epi_score_all(ds.handle, order, _dptr(out)))
    return out


def unrank(ds: Dataset, order: int, ranks):
    """Device combinations (int32 [count, order]) of device int64 ranks."""
    import torch
    ranks = ranks.contiguous()
    out = torch.empty((ranks.numel(), order), dtype=torch.int32, device=ranks.device)
    _check(load().epi_unrank(ds.handle, order, _dptr(ranks), ranks.numel(), _dptr(out)))
    return out


def features5(ds: Dataset, s1, s2, s3, combs, s4=None):
    """25 features of device 5-sets combs (int32 [count, 5]); 30 with the
    order-4 table s4."""
    import torch
    combs = combs.contiguous()
    X = torch.empty((combs.shape[0], 25 if s4 is None else 30), dtype=torch.float32, device=combs.device)
    _check(load().epi_features5(ds.handle, _dptr(s1), _dptr(s2), _dptr(s3), None if s4 is None else _dptr(s4),
                                _dptr(combs), combs.shape[0], _dptr(X)))
    return X


def candidates5(ds: Dataset, triples, first: int, count: int, s3=None):
    """Candidates [first, first + count) of the triples-plus-pair space
    (int32 [count, 5] on the device); with the order-3 table s3, also the
    keep mask (uint8 [count]) that marks each set once."""
    import torch
    triples = triples.contiguous()
    out = torch.empty((count, 5), dtype=torch.int32, device=triples.device)
    keep = None if s3 is None else torch.empty(count, dtype=torch.uint8, device=triples.device)
    _check(load().epi_candidates5(ds.handle, _dptr(triples), triples.shape[0], first, count, _dptr(out),
                                  None if s3 is None else _dptr(s3), None if keep is None else _dptr(keep)))
    return out if s3 is None else (out, keep)


def score5(ds: Dataset, combs):
    """Exact FP32 MI of device order-5 sets (int32 [count, 5]), tables
    counted in registers (float32 [count] on the device)."""
    import torch
    combs = combs.contiguous()
    out = torch.empty(combs.shape[0], dtype=torch.float32, device=combs.device)
    _check(load().epi_score5(ds.handle, _dptr(combs), combs.shape[0], _dptr(out)))
    return out


def lookup(ds: Dataset, order: int, table, combs):
    """table[rank(combs[i])] for device combinations (float32 [count])."""
    import torch
    combs = combs.contiguous()
    out = torch.empty(combs.shape[0], dtype=torch.float32, device=combs.device)
    _check(load().epi_lookup(ds.handle, order, _dptr(table), _dptr(combs), combs.shape[0], _dptr(out)))
    return out


def topk(ctx: Context, scores, k: int, keep=None):
    """(values, indices) of the k largest device floats, ties by index,
    entries with keep == 0 skipped."""
    import torch
    k = min(k, scores.numel())
    vals = torch.empty(k, dtype=torch.float32, device=scores.device)
    idx = torch.empty(k, dtype=torch.int64, device=scores.device)
    n = torch.zeros(1, dtype=torch.int32, device=scores.device)
    _check(load().epi_topk(ctx.handle, _dptr(scores), None if keep is None else _dptr(keep), scores.numel(), k,
                           _dptr(vals), _dptr(idx), _dptr(n)))
    m = int(n.item())
    return vals[:m], idx[:m]


def heuristic5(ctx: Context, X):
    """Network-free ranking score of feature rows (sum of the three-way
    log-scores of 25-column rows, of the four-way ones of 30-column rows)."""
    import torch
    X = X.contiguous()
    out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    _check(load().epi_heuristic5(ctx.handle, _dptr(X), X.shape[0], X.shape[1], _dptr(out)))
    return out


class MLP:
    """The proposer network (see epi_mlp_create)."""

    def __init__(self, ctx: Context, n_in: int = 25, hidden: int = 256, seed: int = 1):
        self.ctx = ctx
        self.n_in, self.hidden = n_in, hidden
        h = C.c_void_p()
        _check(load().epi_mlp_create(ctx.handle, n_in, hidden, seed, C.byref(h)))
        self._h = h
        self.n_params = int(load().epi_mlp_num_params(h))

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(load().epi_mlp_get_params(self._h, _np_ptr(out)))
        return out

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        assert theta.size == self.n_params
        _check(load().epi_mlp_set_params(self._h, _np_ptr(theta)))

    def forward(self, X):
        import torch
        X = X.contiguous()
        y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        _check(load().epi_mlp_forward(self._h, _dptr(X), X.shape[0], _dptr(y)))
        return y

    def gradients(self, X, t):
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = C.c_float(0.0)
        _check(load().epi_mlp_gradients(self._h, _dptr(X.contiguous()), _dptr(t.contiguous()), X.shape[0],
                                         _np_ptr(g), C.byref(loss)))
        return g, loss.value

    def train_step(self, X, t, lr: float, wd: float) -> float:
        loss = C.c_float(0.0)
        _check(load().epi_mlp_train_step(self._h, _dptr(X.contiguous()), _dptr(t.contiguous()), X.shape[0],
                                          lr, wd, C.byref(loss)))
        return loss.value

    def set_forward_path(self, path: str):
        """'auto', 'cuda_cores' or 'tensor_cores' for forward()."""
        _check(load().epi_mlp_set_forward_path(self._h, {"auto": 0, "cuda_cores": 1, "tensor_cores": 2}[path]))

    def input_norm(self) -> tuple[np.ndarray, np.ndarray]:
        shift = np.zeros(self.n_in, dtype=np.float32)
        scale = np.zeros(self.n_in, dtype=np.float32)
        _check(load().epi_mlp_get_input_norm(self._h, _np_ptr(shift), _np_ptr(scale)))
        return shift, scale

    def set_input_norm(self, shift, scale):
        shift = np.ascontiguousarray(shift, dtype=np.float32)
        scale = np.ascontiguousarray(scale, dtype=np.float32)
        assert shift.size == self.n_in and scale.size == self.n_in
        _check(load().epi_mlp_set_input_norm(self._h, _np_ptr(shift), _np_ptr(scale)))

    def save(self, path: str):
        """Flat little-endian file: int32 n_in, hidden; float32 parameters
        (epi_mlp_create's order), input shift [n_in], input scale [n_in]."""
        shift, scale = self.input_norm()
        with open(path, "wb") as f:
            np.array([self.n_in, self.hidden], dtype="<i4").tofile(f)
            self.params().astype("<f4").tofile(f)
            shift.astype("<f4").tofile(f)
            scale.astype("<f4").tofile(f)

    def load_file(self, path: str):
        with open(path, "rb") as f:
            hdr = np.fromfile(f, dtype="<i4", count=2)
            if tuple(hdr) != (self.n_in, self.hidden):
                raise ValueError(f"network shape {tuple(hdr)} does not match {(self.n_in, self.hidden)}")
            theta = np.fromfile(f, dtype="<f4", count=self.n_params)
            norm = np.fromfile(f, dtype="<f4", count=2 * self.n_in)
            if theta.size != self.n_params or norm.size != 2 * self.n_in:
                raise ValueError("truncated network file")
            self.set_params(theta)
            self.set_input_norm(norm[:self.n_in], norm[self.n_in:])

    def close(self):
        if getattr(self, "_h", None):
            load().epi_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def proposer_search(ds: Dataset, net: "MLP | None", top_triples: int, budget: int, top_n: int,
                    chunk: int = 0, with_counts: bool = False,
                    quad_features: bool | None = None) -> tuple[SearchResult, dict]:
    """Order-5 proposals ranked by `net` (None: the network-free heuristic),
    re-scored exactly (see epi_proposer_search).  quad_features (default: the
    network takes 30 inputs) selects the 30 features with four-way scores."""
    if quad_features is None:
        quad_features = net is not None and net.n_in == 30
    out = np.zeros(top_n, dtype=RESULT_DTYPE)
    counts = np.zeros((top_n, 2, 243), dtype=np.uint32) if with_counts else None
    n_out = C.c_int(0)
    opts = ProposerOpts(top_triples, budget, top_n, chunk, 1 if quad_features else 0)
    stats = ProposerStats()
    _check(load().epi_proposer_search(ds.handle, None if net is None else net._h, C.byref(opts), _np_ptr(out),
                                      _np_ptr(counts) if with_counts else None, C.byref(n_out), C.byref(stats)))
    n = n_out.value
    st = {f: getattr(stats, f) for f, _ in ProposerStats._fields_}
    return SearchResult(out[:n], counts[:n] if with_counts else None, 5), st


TARGETS = {"log_mi": 0, "top_membership": 1}


def proposer_train(net: "MLP", datasets, top_triples: int, epochs: int, batch: int, lr: float, wd: float = 0.0,
                   tail_fraction: float = 0.5, seed: int = 1, target: str = "log_mi") -> np.ndarray:
    """Fit `net` on exhaustive order-5 labels of `datasets` (see
    epi_proposer_train); returns the mean sampled batch loss per epoch."""
    arr = (C.c_void_p * len(datasets))(*[d.handle for d in datasets])
    losses = np.zeros(epochs, dtype=np.float32)
    opts = TrainOpts(top_triples, epochs, batch, lr, wd, tail_fraction, seed, TARGETS[target])
    _check(load().epi_proposer_train(net._h, arr, len(datasets), C.byref(opts), _np_ptr(losses)))
    return losses
