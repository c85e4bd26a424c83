"""Thin ctypes binding of the C ABI in include/tc.h (argument marshalling
only: every step of the contraction runs in the CUDA library).

The functions carry the C names (``tc_plan_create``, ``tc_execute``, ...);
``Plan`` wraps a plan handle.  Device buffers are passed as integers or as
objects with ``data_ptr()`` (torch tensors); streams as integers or objects
with ``cuda_stream`` / ``stream_id`` (torch streams).  The library is loaded
on first use; a missing library raises ``RuntimeError`` -- there is no
fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtc.so")

TC_SUCCESS = 0
STATUS_NAMES = {
    0: "TC_SUCCESS", 1: "TC_ERROR_INVALID_SPEC", 2: "TC_ERROR_INVALID_EXTENT",
    3: "TC_ERROR_INVALID_STRIDE", 4: "TC_ERROR_UNSUPPORTED_DTYPE",
    5: "TC_ERROR_INVALID_ALGORITHM", 6: "TC_ERROR_OUT_OF_MEMORY",
    7: "TC_ERROR_CUDA", 8: "TC_ERROR_TIMEOUT", 9: "TC_ERROR_INVALID_ARGUMENT",
    10: "TC_ERROR_ADMISSION",
}
DTYPES = {"f64": 0, "f32": 1, "tf32": 2, "bf16": 3, "f16": 4, "bf16x3": 5, "tf32x3": 6, "e4m3": 7}
KERNELS = ("dot", "axpy", "gemv", "ger", "gemm", "gett")


class TcError(RuntimeError):
    def __init__(self, status, where, message=""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}"
                         + (f" ({message})" if message else ""))


class tc_algorithm(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_int32),
        ("name", ctypes.c_char * 32),
        ("kernel", ctypes.c_int32),
        ("n_loops", ctypes.c_int32),
        ("loops", ctypes.c_char * 8),
        ("n_kernel_indices", ctypes.c_int32),
        ("kernel_indices", ctypes.c_char * 4),
        ("copy_mask", ctypes.c_uint32),
        ("copy_level", ctypes.c_int32 * 3),
        ("n_phases", ctypes.c_int32),
    ]


class tc_pred_case(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("depth", ctypes.c_int32), ("count", ctypes.c_int64),
                ("omit", ctypes.c_int32), ("n_items", ctypes.c_int32)]


class tc_setup_item(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("operand", ctypes.c_int32), ("size", ctypes.c_int64)]


class tc_batch_tuning(ctypes.Structure):
    _fields_ = [("m_log2", ctypes.c_int32), ("k_log2", ctypes.c_int32), ("n_class", ctypes.c_int32),
                ("problems", ctypes.c_int32), ("candidates", ctypes.c_int32), ("tile_m", ctypes.c_int32),
                ("tile_n", ctypes.c_int32), ("k_chunk", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("seconds_best", ctypes.c_double),
                ("seconds_rule", ctypes.c_double), ("seconds_fixed", ctypes.c_double)]


class tc_chain_variant(ctypes.Structure):
    _fields_ = [("first", ctypes.c_int32 * 2), ("third", ctypes.c_int32), ("sliced", ctypes.c_char),
                ("slices", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64), ("flops", ctypes.c_double),
                ("algorithm", ctypes.c_int32 * 2), ("predicted_seconds", ctypes.c_double)]


class tc_server_report(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("admission_stalls", ctypes.c_int64), ("peak_inflight", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("flops_served", ctypes.c_double),
                ("span_seconds", ctypes.c_double), ("p50_seconds", ctypes.c_double),
                ("p99_seconds", ctypes.c_double), ("max_seconds", ctypes.c_double),
                ("batches", ctypes.c_int64), ("max_batch", ctypes.c_int64)]


_lib = None

# name -> (restype, argtypes); mirrors include/tc.h
_VP, _I64P, _I32P = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)
SIGNATURES = {
    "tc_plan_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_char_p, _I64P, _I64P, ctypes.c_int]),
    "tc_plan_destroy": (ctypes.c_int, [_VP]),
    "tc_algorithm_count": (ctypes.c_int, [_VP, _I32P]),
    "tc_enumerate_algorithms": (ctypes.c_int, [_VP, ctypes.POINTER(tc_algorithm), ctypes.c_int32, _I32P]),
    "tc_plan_select": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "tc_plan_selected": (ctypes.c_int, [_VP, _I32P]),
    "tc_algorithm_workspace": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "tc_execute": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "tc_execute_no_alloc": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "tc_execute_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "tc_plan_device_status": (ctypes.c_int, [_VP]),
    "tc_plan_flops": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "tc_plan_set_split": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "tc_plan_set_gett_tile": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "tc_plan_set_gett_tma": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "tc_plan_set_gett_pack": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "tc_plan_set_compensation": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "tc_plan_set_gett_pair": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "tc_plan_set_split_accumulators": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "tc_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, _VP]),
    "tc_access_distances": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _I64P]),
    "tc_prediction_cases": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_int64, ctypes.POINTER(tc_pred_case), ctypes.c_int32, _I32P]),
    "tc_setup_list": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(tc_setup_item),
                                     ctypes.c_int32, _I32P]),
    "tc_predict": (ctypes.c_int, [_VP, _I32P, ctypes.c_int32, _VP, _VP, _VP,
                                  ctypes.POINTER(ctypes.c_double), _VP]),
    "tc_plan_select_best": (ctypes.c_int, [_VP, _I32P]),
    "tc_autotune": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _I32P, _I32P]),
    "tc_plan_get_gett_config": (ctypes.c_int, [_VP, _I32P, _I32P, _I32P, _I32P]),
    "tc_tuning_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
    "tc_tuning_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
    "tc_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_char_p, ctypes.c_int32, _I64P, ctypes.c_int]),
    "tc_batch_destroy": (ctypes.c_int, [_VP]),
    "tc_batch_set_tiles": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "tc_batch_set_operands": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    "tc_batch_prepare": (ctypes.c_int, [_VP]),
    "tc_batch_execute": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, _VP]),
    "tc_batch_info": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), _I64P, _I64P]),
    "tc_batch_device_status": (ctypes.c_int, [_VP]),
    "tc_batch_autotune": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, ctypes.POINTER(tc_batch_tuning), ctypes.c_int32,
                                         _I32P]),
    "tc_batch_config": (ctypes.c_int, [_VP, _I32P, _I32P, _I32P, _I32P]),
    "tc_batch_problem_tiles": (ctypes.c_int, [_VP, ctypes.c_int32, _I32P, _I32P, _I32P]),
    "tc_chain_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_char_p, _I64P, ctypes.c_int]),
    "tc_chain_destroy": (ctypes.c_int, [_VP]),
    "tc_chain_variants": (ctypes.c_int, [_VP, ctypes.POINTER(tc_chain_variant), ctypes.c_int32, _I32P]),
    "tc_chain_set_workspace_limit": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "tc_chain_predict": (ctypes.c_int, [_VP, ctypes.c_int32, _VP]),
    "tc_chain_select": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "tc_chain_selected": (ctypes.c_int, [_VP, _I32P]),
    "tc_chain_execute": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "tc_chain_device_status": (ctypes.c_int, [_VP]),
    "tc_server_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]),
    "tc_server_submit": (ctypes.c_int, [_VP, ctypes.c_char_p, _I64P, ctypes.c_int, _VP, _VP, _VP, _I64P]),
    "tc_server_poll": (ctypes.c_int, [_VP, ctypes.c_int64, _I32P, ctypes.POINTER(ctypes.c_double)]),
    "tc_server_wait": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_double]),
    "tc_server_stats": (ctypes.c_int, [_VP, ctypes.POINTER(tc_server_report)]),
    "tc_server_destroy": (ctypes.c_int, [_VP]),
    "tc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tc_last_error": (ctypes.c_char_p, []),
}


def load(path=LIB_PATH):
    """Load libtc.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libtc.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status, where):
    if status != TC_SUCCESS:
        msg = load().tc_last_error().decode(errors="replace")
        raise TcError(status, where, msg)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    for attr in ("cuda_stream", "stream_id"):
        if hasattr(s, attr):
            return int(getattr(s, attr))
    return int(s)


def _i64(vals):
    if vals is None:
        return None
    vals = [int(v) for v in vals]
    return (ctypes.c_int64 * len(vals))(*vals)


def _scalar(value, dtype):
    return ctypes.c_double(value) if dtype == "f64" else ctypes.c_float(value)


# ---------------------------------------------------------------- C names
def tc_plan_create(spec, extents, strides=None, dtype="f64"):
    h = ctypes.c_void_p()
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    _check(load().tc_plan_create(ctypes.byref(h), spec.encode(), _i64(extents),
                                 _i64(strides), dt), "tc_plan_create")
    return h


def tc_plan_destroy(plan):
    _check(load().tc_plan_destroy(plan), "tc_plan_destroy")


def tc_enumerate_algorithms(plan):
    n = ctypes.c_int32()
    _check(load().tc_enumerate_algorithms(plan, None, 0, ctypes.byref(n)), "tc_enumerate_algorithms")
    buf = (tc_algorithm * n.value)()
    _check(load().tc_enumerate_algorithms(plan, buf, n.value, ctypes.byref(n)), "tc_enumerate_algorithms")
    out = []
    for a in buf:
        out.append({
            "id": a.id,
            "name": a.name.decode(),
            "kernel": KERNELS[a.kernel],
            "loops": tuple(chr(c) for c in a.loops[:a.n_loops]),
            "kernel_indices": tuple(chr(c) for c in a.kernel_indices[:a.n_kernel_indices]),
            "copy_mask": a.copy_mask,
            "copy_level": tuple(a.copy_level),
            "n_phases": a.n_phases,
        })
    return out


def tc_plan_select(plan, alg_id):
    _check(load().tc_plan_select(plan, int(alg_id)), "tc_plan_select")


def tc_plan_selected(plan):
    v = ctypes.c_int32()
    _check(load().tc_plan_selected(plan, ctypes.byref(v)), "tc_plan_selected")
    return v.value


def tc_algorithm_workspace(plan, alg_id):
    v = ctypes.c_size_t()
    _check(load().tc_algorithm_workspace(plan, int(alg_id), ctypes.byref(v)), "tc_algorithm_workspace")
    return v.value


def tc_execute(plan, alpha, A, B, beta, C, stream=None, dtype="f64"):
    a, b = _scalar(alpha, dtype), _scalar(beta, dtype)
    _check(load().tc_execute(plan, ctypes.addressof(a), _ptr(A), _ptr(B), ctypes.addressof(b),
                             _ptr(C), _stream(stream)), "tc_execute")


def tc_execute_host(plan, alpha, hA, hB, beta, hC, stream=None, dtype="f64"):
    """Host buffers (pointers or pinned CPU tensors); enqueued on stream."""
    a, b = _scalar(alpha, dtype), _scalar(beta, dtype)
    _check(load().tc_execute_host(plan, ctypes.addressof(a), _ptr(hA), _ptr(hB), ctypes.addressof(b),
                                  _ptr(hC), _stream(stream)), "tc_execute_host")


def tc_execute_no_alloc(plan, alpha, A, B, beta, C, stream=None, dtype="f64"):
    a, b = _scalar(alpha, dtype), _scalar(beta, dtype)
    _check(load().tc_execute_no_alloc(plan, ctypes.addressof(a), _ptr(A), _ptr(B), ctypes.addressof(b),
                                      _ptr(C), _stream(stream)), "tc_execute_no_alloc")


def tc_plan_device_status(plan):
    _check(load().tc_plan_device_status(plan), "tc_plan_device_status")


def tc_plan_set_split(plan, products):
    _check(load().tc_plan_set_split(plan, int(products)), "tc_plan_set_split")


def tc_plan_set_gett_tile(plan, width):
    _check(load().tc_plan_set_gett_tile(plan, int(width)), "tc_plan_set_gett_tile")


def tc_plan_set_gett_tma(plan, enable):
    _check(load().tc_plan_set_gett_tma(plan, int(enable)), "tc_plan_set_gett_tma")


def tc_plan_set_gett_pack(plan, mode):
    _check(load().tc_plan_set_gett_pack(plan, int(mode)), "tc_plan_set_gett_pack")


def tc_selftest_bounded_wait(limit_ns, signal, stream=None):
    """Runs the bounded-wait self-test; returns the status (no exception)."""
    return load().tc_selftest_bounded_wait(int(limit_ns), int(signal), _stream(stream))


def tc_plan_set_compensation(plan, chunk):
    _check(load().tc_plan_set_compensation(plan, int(chunk)), "tc_plan_set_compensation")


def tc_plan_set_gett_pair(plan, enable):
    _check(load().tc_plan_set_gett_pair(plan, int(enable)), "tc_plan_set_gett_pair")


def tc_plan_set_split_accumulators(plan, enable):
    _check(load().tc_plan_set_split_accumulators(plan, int(enable)), "tc_plan_set_split_accumulators")


def tc_plan_flops(plan):
    v = ctypes.c_double()
    _check(load().tc_plan_flops(plan, ctypes.byref(v)), "tc_plan_flops")
    return v.value


OPERAND_NAMES = ("A", "B", "C")
CASE_KINDS = ("steady", "miss", "first")


def tc_access_distances(plan, alg_id, granularity=0, elem_size=1):
    out = (ctypes.c_int64 * 3)()
    _check(load().tc_access_distances(plan, int(alg_id), int(granularity), int(elem_size), out),
           "tc_access_distances")
    return dict(zip(OPERAND_NAMES, list(out)))


def tc_prediction_cases(plan, alg_id, granularity=0, elem_size=1, cache_size=1 << 20, line_size=8):
    n = ctypes.c_int32()
    args = (plan, int(alg_id), int(granularity), int(elem_size), int(cache_size), int(line_size))
    _check(load().tc_prediction_cases(*args, None, 0, ctypes.byref(n)), "tc_prediction_cases")
    buf = (tc_pred_case * n.value)()
    _check(load().tc_prediction_cases(*args, buf, n.value, ctypes.byref(n)), "tc_prediction_cases")
    return [{"kind": CASE_KINDS[c.kind], "depth": c.depth, "count": c.count, "omit": bool(c.omit),
             "n_items": c.n_items} for c in buf]


def tc_setup_list(plan, alg_id, case_index, granularity=0, elem_size=1, cache_size=1 << 20, line_size=8):
    """Setup list as [("op", "A"|"B"|"C", size) | ("remote", size)]."""
    n = ctypes.c_int32()
    args = (plan, int(alg_id), int(granularity), int(case_index), int(elem_size), int(cache_size),
            int(line_size))
    _check(load().tc_setup_list(*args, None, 0, ctypes.byref(n)), "tc_setup_list")
    buf = (tc_setup_item * n.value)()
    _check(load().tc_setup_list(*args, buf, n.value, ctypes.byref(n)), "tc_setup_list")
    return [("op", OPERAND_NAMES[i.operand], i.size) if i.kind == 0 else ("remote", i.size) for i in buf]


def tc_predict(plan, alg_ids=None, A=None, B=None, C=None, stream=None):
    """Predicted seconds per algorithm (a list aligned with alg_ids, or with
    every algorithm when alg_ids is None)."""
    if alg_ids is None:
        n = ctypes.c_int32()
        _check(load().tc_algorithm_count(plan, ctypes.byref(n)), "tc_algorithm_count")
        ids, count = None, n.value
    else:
        ids = (ctypes.c_int32 * len(alg_ids))(*[int(x) for x in alg_ids])
        count = len(alg_ids)
    out = (ctypes.c_double * count)()
    _check(load().tc_predict(plan, ids, count, _ptr(A), _ptr(B), _ptr(C), out, _stream(stream)),
           "tc_predict")
    return list(out)


def tc_plan_select_best(plan):
    v = ctypes.c_int32()
    _check(load().tc_plan_select_best(plan, ctypes.byref(v)), "tc_plan_select_best")
    return v.value


def tc_autotune(plan, A=None, B=None, C=None, stream=None):
    w, t = ctypes.c_int32(), ctypes.c_int32()
    _check(load().tc_autotune(plan, _ptr(A), _ptr(B), _ptr(C), _stream(stream), ctypes.byref(w),
                              ctypes.byref(t)), "tc_autotune")
    return w.value, t.value


def tc_tuning_cache_save(path):
    _check(load().tc_tuning_cache_save(str(path).encode()), "tc_tuning_cache_save")


def tc_tuning_cache_load(path):
    _check(load().tc_tuning_cache_load(str(path).encode()), "tc_tuning_cache_load")


class Batch:
    """Owns a tc_batch: many independent contractions in one launch."""

    def __init__(self, spec, extents, dtype="f32"):
        rows = [list(map(int, r)) for r in extents]
        flat = [x for r in rows for x in r]
        self.dtype = dtype
        self.count = len(rows)
        h = ctypes.c_void_p()
        _check(load().tc_batch_create(ctypes.byref(h), spec.encode(), len(rows), _i64(flat),
                                      DTYPES[dtype]), "tc_batch_create")
        self.handle = h

    def set_tiles(self, policy):
        _check(load().tc_batch_set_tiles(self.handle, int(policy)), "tc_batch_set_tiles")

    def set_operands(self, A, B, C):
        arr = lambda xs: (ctypes.c_void_p * len(xs))(*[_ptr(x) for x in xs])
        _check(load().tc_batch_set_operands(self.handle, arr(A), arr(B), arr(C)), "tc_batch_set_operands")

    def prepare(self):
        _check(load().tc_batch_prepare(self.handle), "tc_batch_prepare")

    def execute(self, alpha=1.0, beta=0.0, per_problem=False, stream=None):
        a, b = _scalar(alpha, self.dtype), _scalar(beta, self.dtype)
        _check(load().tc_batch_execute(self.handle, ctypes.addressof(a), ctypes.addressof(b),
                                       1 if per_problem else 0, _stream(stream)), "tc_batch_execute")

    def info(self):
        f, t, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().tc_batch_info(self.handle, ctypes.byref(f), ctypes.byref(t), ctypes.byref(b)),
               "tc_batch_info")
        return {"flops": f.value, "tiles": t.value, "bytes": b.value}

    def device_status(self):
        _check(load().tc_batch_device_status(self.handle), "tc_batch_device_status")

    def autotune(self, stream=None, reps=5):
        """Per shape class: the fastest (tile shape, K chunk) by timing; leaves policy 2 selected."""
        cap = 9 * 8 * 3  # ceil(log2 M) <= 8, ceil(log2 K) <= 7, three N buckets
        buf = (tc_batch_tuning * cap)()
        n = ctypes.c_int32()
        _check(load().tc_batch_autotune(self.handle, _stream(stream), int(reps), buf, cap, ctypes.byref(n)),
               "tc_batch_autotune")
        return [{f: getattr(buf[i], f) for f, _ in tc_batch_tuning._fields_} for i in range(min(n.value, cap))]

    def config(self):
        v = [ctypes.c_int32() for _ in range(4)]
        _check(load().tc_batch_config(self.handle, *[ctypes.byref(x) for x in v]), "tc_batch_config")
        return {"policy": v[0].value, "stages": v[1].value, "tile_n": v[2].value,
                "kernel": ["simt", "gett", "stream"][v[3].value]}

    def problem_tiles(self, q):
        m, n, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().tc_batch_problem_tiles(self.handle, int(q), ctypes.byref(m), ctypes.byref(n), ctypes.byref(k)),
               "tc_batch_problem_tiles")
        return m.value, n.value, k.value

    def close(self):
        if self.handle is not None and _lib is not None:
            load().tc_batch_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Chain:
    """Owns a tc_chain: D = X Y Z through an intermediate, order and slicing
    chosen by flops or by prediction."""

    def __init__(self, spec, extents, dtype="f64"):
        h = ctypes.c_void_p()
        _check(load().tc_chain_create(ctypes.byref(h), spec.encode(), _i64([int(e) for e in extents]),
                                      DTYPES[dtype]), "tc_chain_create")
        self.handle = h
        self.dtype = dtype

    def variants(self):
        n = ctypes.c_int32()
        _check(load().tc_chain_variants(self.handle, None, 0, ctypes.byref(n)), "tc_chain_variants")
        buf = (tc_chain_variant * max(1, n.value))()
        _check(load().tc_chain_variants(self.handle, buf, n.value, ctypes.byref(n)), "tc_chain_variants")
        out = []
        for v in buf[:n.value]:
            out.append({"first": (v.first[0], v.first[1]), "third": v.third,
                        "sliced": v.sliced.decode() if v.sliced != b"\x00" else None, "slices": v.slices,
                        "workspace_bytes": v.workspace_bytes, "flops": v.flops,
                        "algorithm": (v.algorithm[0], v.algorithm[1]), "predicted_seconds": v.predicted_seconds})
        return out

    def set_workspace_limit(self, nbytes):
        _check(load().tc_chain_set_workspace_limit(self.handle, int(nbytes)), "tc_chain_set_workspace_limit")

    def predict(self, all_algorithms=False, stream=None):
        _check(load().tc_chain_predict(self.handle, 1 if all_algorithms else 0, _stream(stream)), "tc_chain_predict")

    def select(self, variant=-1):
        _check(load().tc_chain_select(self.handle, int(variant)), "tc_chain_select")

    def selected(self):
        v = ctypes.c_int32()
        _check(load().tc_chain_selected(self.handle, ctypes.byref(v)), "tc_chain_selected")
        return v.value

    def execute(self, X, Y, Z, D, alpha=1.0, beta=0.0, stream=None):
        sd = "f64" if self.dtype == "f64" else "f32"
        a, b = _scalar(alpha, sd), _scalar(beta, sd)
        _check(load().tc_chain_execute(self.handle, ctypes.addressof(a), _ptr(X), _ptr(Y), _ptr(Z),
                                       ctypes.addressof(b), _ptr(D), _stream(stream)), "tc_chain_execute")

    def device_status(self):
        _check(load().tc_chain_device_status(self.handle), "tc_chain_device_status")

    def close(self):
        if self.handle is not None and _lib is not None:
            load().tc_chain_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owns a tc_server (continuous batching of contraction requests)."""

    def __init__(self, budget_bytes=40 << 30, slots=32, streams=8):
        h = ctypes.c_void_p()
        _check(load().tc_server_create(ctypes.byref(h), int(budget_bytes), int(slots), int(streams)),
               "tc_server_create")
        self.handle = h

    def submit(self, spec, extents, dtype, A, B, C=None):
        rid = ctypes.c_int64()
        _check(load().tc_server_submit(self.handle, spec.encode(), _i64(extents), DTYPES[dtype], _ptr(A),
                                       _ptr(B), _ptr(C), ctypes.byref(rid)), "tc_server_submit")
        return rid.value

    def poll(self, rid):
        done, lat = ctypes.c_int32(), ctypes.c_double()
        st = load().tc_server_poll(self.handle, int(rid), ctypes.byref(done), ctypes.byref(lat))
        if done.value:
            _check(st, "tc_server_poll")
        return bool(done.value), lat.value

    def wait(self, rid, timeout=60.0):
        _check(load().tc_server_wait(self.handle, int(rid), float(timeout)), "tc_server_wait")

    def stats(self):
        s = tc_server_report()
        _check(load().tc_server_stats(self.handle, ctypes.byref(s)), "tc_server_stats")
        return {name: getattr(s, name) for name, _ in tc_server_report._fields_}

    def close(self):
        if self.handle is not None and _lib is not None:
            load().tc_server_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_status_string(status):
    return load().tc_status_string(int(status)).decode()


# ---------------------------------------------------------------- convenience
class Plan:
    """Owns one plan handle (destroyed on close / garbage collection)."""

    def __init__(self, spec, extents, strides=None, dtype="f64"):
        self.spec, self.extents, self.dtype = spec, list(extents), dtype
        self.handle = tc_plan_create(spec, extents, strides, dtype)

    def algorithms(self):
        return tc_enumerate_algorithms(self.handle)

    def select(self, alg_id):
        tc_plan_select(self.handle, alg_id)

    @property
    def selected(self):
        return tc_plan_selected(self.handle)

    def workspace(self, alg_id):
        return tc_algorithm_workspace(self.handle, alg_id)

    def execute(self, A, B, C, alpha=1.0, beta=0.0, stream=None):
        tc_execute(self.handle, alpha, A, B, beta, C, stream, self.dtype)

    def execute_host(self, hA, hB, hC, alpha=1.0, beta=0.0, stream=None):
        tc_execute_host(self.handle, alpha, hA, hB, beta, hC, stream, self.dtype)

    def set_split(self, products):
        tc_plan_set_split(self.handle, products)

    def set_gett_tile(self, width):
        tc_plan_set_gett_tile(self.handle, width)

    def set_gett_tma(self, enable):
        tc_plan_set_gett_tma(self.handle, enable)

    def set_gett_pack(self, mode):
        tc_plan_set_gett_pack(self.handle, mode)

    def set_compensation(self, chunk):
        tc_plan_set_compensation(self.handle, chunk)

    def set_gett_pair(self, enable):
        tc_plan_set_gett_pair(self.handle, enable)

    def set_split_accumulators(self, enable):
        tc_plan_set_split_accumulators(self.handle, enable)

    def predict(self, alg_ids=None, A=None, B=None, C=None, stream=None):
        return tc_predict(self.handle, alg_ids, A, B, C, stream)

    def select_best(self):
        return tc_plan_select_best(self.handle)

    def autotune(self, A=None, B=None, C=None, stream=None):
        return tc_autotune(self.handle, A, B, C, stream)

    def gett_config(self):
        v = [ctypes.c_int32() for _ in range(4)]
        _check(load().tc_plan_get_gett_config(self.handle, *[ctypes.byref(x) for x in v]),
               "tc_plan_get_gett_config")
        return {"width": v[0].value, "tma": v[1].value, "pair": v[2].value, "pack": v[3].value}

    def device_status(self):
        tc_plan_device_status(self.handle)

    @property
    def flops(self):
        return tc_plan_flops(self.handle)

    def close(self):
        if self.handle is not None and _lib is not None:
            tc_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
