"""ctypes declarations of the C ABI in include/tz.h (argument marshalling only).

Loading fails loudly when libtz.so has not been built: there is no other
implementation to fall back to.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtz.so")

TZ_OK, TZ_EINVAL, TZ_ENOMEM, TZ_EHBM_ADMIT, TZ_ECUDA, TZ_ETIMEOUT, TZ_EUNSUPPORTED, TZ_EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
TZ_LATTICE_GRID, TZ_LATTICE_BRISTLECONE = 0, 1
TZ_C64_SIMT, TZ_TF32X3, TZ_BF16X3, TZ_C128_SIMT, TZ_FP16X3 = 0, 1, 2, 3, 4
PRECISIONS = {"c64": TZ_C64_SIMT, "tf32x3": TZ_TF32X3, "bf16x3": TZ_BF16X3, "c128": TZ_C128_SIMT,
              "fp16x3": TZ_FP16X3}

_ERR_NAMES = {TZ_EINVAL: "TZ_EINVAL", TZ_ENOMEM: "TZ_ENOMEM", TZ_EHBM_ADMIT: "TZ_EHBM_ADMIT", TZ_ECUDA: "TZ_ECUDA",
              TZ_ETIMEOUT: "TZ_ETIMEOUT", TZ_EUNSUPPORTED: "TZ_EUNSUPPORTED", TZ_EBUSY: "TZ_EBUSY"}


class TzError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class tz_lattice(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("rows", ctypes.c_int), ("cols", ctypes.c_int), ("n_qubits", ctypes.c_int)]


class tz_network_opts(ctypes.Structure):
    _fields_ = [("batch_log2", ctypes.c_int), ("n_open", ctypes.c_int), ("open_qubits", ctypes.POINTER(ctypes.c_int32))]


class tz_path_opts(ctypes.Structure):
    _fields_ = [("restarts", ctypes.c_int), ("seed", ctypes.c_uint64), ("log2_max_intermediate", ctypes.c_int),
                ("precision", ctypes.c_int), ("algorithm", ctypes.c_int), ("reconfigure", ctypes.c_int)]


class tz_plan_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("device", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("small_log2", ctypes.c_int), ("use_graph", ctypes.c_int), ("max_bitstrings", ctypes.c_int64),
                ("autotune", ctypes.c_int), ("direct_queue", ctypes.c_int)]


class tz_plan_stats(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int), ("n_const_steps", ctypes.c_int), ("n_gemm_steps", ctypes.c_int),
                ("n_permutes", ctypes.c_int), ("n_launches_per_group", ctypes.c_int), ("k", ctypes.c_int),
                ("batch_log2", ctypes.c_int), ("max_log2", ctypes.c_int), ("flops_per_group", ctypes.c_double),
                ("gemm_flops_per_group", ctypes.c_double), ("bytes_per_group", ctypes.c_double),
                ("permute_bytes_per_group", ctypes.c_double), ("workspace_bytes", ctypes.c_size_t),
                ("const_bytes", ctypes.c_size_t), ("scratch_bytes", ctypes.c_size_t), ("const_flops", ctypes.c_double),
                ("bind_ms", ctypes.c_double), ("n_tuned_steps", ctypes.c_int), ("n_open", ctypes.c_int)]


PROFILE_KINDS = ("leaves", "direct", "permute", "gemm_simt", "gemm_tc", "accumulate", "gemm_skinny", "gemm_dot")


class tz_plan_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 8), ("ms", ctypes.c_double * 8), ("flops", ctypes.c_double * 8),
                ("bytes", ctypes.c_double * 8)]


class tz_server_opts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_inflight", ctypes.c_int), ("device", ctypes.c_int),
                ("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t), ("wait_admit", ctypes.c_int),
                ("chunk_ms", ctypes.c_double)]


P = ctypes.c_void_p
PP = ctypes.POINTER(ctypes.c_void_p)
I32P = ctypes.POINTER(ctypes.c_int32)
U8P = ctypes.POINTER(ctypes.c_uint8)
F64P = ctypes.POINTER(ctypes.c_double)
c_int, c_size_t, c_int64, c_uint64, c_double = ctypes.c_int, ctypes.c_size_t, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double

# name -> (restype, argtypes)
SIGNATURES = {
    "tz_last_error": (ctypes.c_char_p, []),
    "tz_circuit_from_spec": (c_int, [ctypes.c_char_p, c_size_t, PP]),
    "tz_circuit_generate": (c_int, [ctypes.POINTER(tz_lattice), c_int, c_uint64, PP]),
    "tz_circuit_n_qubits": (c_int, [P]),
    "tz_circuit_n_gates": (c_int, [P]),
    "tz_circuit_to_spec": (c_int, [P, ctypes.c_char_p, c_size_t, ctypes.POINTER(c_size_t)]),
    "tz_circuit_destroy": (None, [P]),
    "tz_network_from_circuit": (c_int, [P, ctypes.POINTER(tz_network_opts), PP]),
    "tz_network_n_tensors": (c_int, [P]),
    "tz_network_n_indices": (c_int, [P]),
    "tz_network_index_info": (c_int, [P, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "tz_network_tensor_indices": (c_int, [P, c_int, I32P, c_int, ctypes.POINTER(c_int)]),
    "tz_network_destroy": (None, [P]),
    "tz_path_greedy": (c_int, [P, ctypes.POINTER(tz_path_opts), PP]),
    "tz_tree_from_pairs": (c_int, [P, I32P, c_int, PP]),
    "tz_tree_pairs": (c_int, [P, I32P, c_int, ctypes.POINTER(c_int)]),
    "tz_tree_destroy": (None, [P]),
    "tz_slice_select": (c_int, [P, P, c_int, c_int, I32P, ctypes.POINTER(c_int)]),
    "tz_plan_create": (c_int, [P, P, I32P, c_int, ctypes.POINTER(tz_plan_opts), PP]),
    "tz_plan_stats_get": (c_int, [P, ctypes.POINTER(tz_plan_stats)]),
    "tz_plan_bind_workspace": (c_int, [P, P, c_size_t]),
    "tz_plan_set_slice_range": (c_int, [P, c_int64, c_int64]),
    "tz_plan_sliced_segments": (c_int, [P, I32P, c_int, ctypes.POINTER(c_int)]),
    "tz_plan_describe": (c_int, [P, ctypes.c_char_p, c_size_t, ctypes.POINTER(c_size_t)]),
    "tz_contract_amplitudes": (c_int, [P, U8P, c_int64, F64P]),
    "tz_contract_amplitudes_device": (c_int, [P, P, c_int64, P]),
    "tz_plan_destroy": (None, [P]),
    "tz_plan_profile_enable": (c_int, [P, c_int]),
    "tz_plan_profile_get": (c_int, [P, ctypes.POINTER(tz_plan_profile)]),
    "tz_plan_profile_items": (c_int, [P, F64P, c_int, ctypes.POINTER(c_int)]),
    "tz_server_create": (c_int, [ctypes.POINTER(tz_server_opts), PP]),
    "tz_server_submit": (c_int, [P, P, U8P, c_int64, ctypes.POINTER(c_uint64)]),
    "tz_server_poll": (c_int, [P, c_uint64, F64P, ctypes.POINTER(c_int)]),
    "tz_server_latency": (c_int, [P, F64P, F64P, ctypes.POINTER(c_int64)]),
    "tz_server_destroy": (None, [P]),
    "tz_op_permute": (c_int, [P, P, c_int, I32P, P]),
    "tz_op_cgemm": (c_int, [c_int, c_int64, c_int64, c_int64, c_int64, P, c_int64, P, c_int64, P, c_int64, P,
                            c_size_t, P]),
    "tz_op_cgemm_scratch_bytes": (c_int, [c_int, c_int64, c_int64, c_int64, c_int64, ctypes.POINTER(c_size_t)]),
    "tz_op_accumulate": (c_int, [P, F64P, c_int64, c_double, c_double, P]),
    "tz_op_cgemm_static": (c_int, [c_int, c_int64, c_int64, c_int64, c_int64, P, c_int64, P, c_int64, P, c_int64, P]),
    "tz_plan_status": (c_int, [P]),
    "tz_op_cgemm_status": (c_int, [c_int, P, P]),
    "tz_op_cgemm_static_status": (c_int, [P]),
    "tz_debug_set_wait_limit": (c_int, [c_int64]),
    "tz_debug_stall_tensor_core": (c_int, [c_int]),
    "tz_debug_stall_direct_queue": (c_int, [c_int]),
    "tz_tune_tc_pairs": (c_int, [c_int]),
    "tz_tune_tc_prefetch": (c_int, [c_int]),
    "tz_debug_tune_force_simt": (c_int, [c_int]),
    "tz_tune_preset": (c_int, [c_int, c_int64, c_int64, c_int64, c_int64, c_int, c_int, c_int, c_int]),
    "tz_debug_stream_tile": (c_int, [c_int64, c_int64, c_int64, c_int64, c_int, P, P, P, P, P]),
}

_lib = None


def lib():
    """The loaded library (ctypes.CDLL) with every signature declared."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_1907_11217_gb300.build` "
                              "(needs nvcc); the library has no fallback implementation")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc):
    if rc is not None and rc < 0:
        raise TzError(rc, lib().tz_last_error().decode(errors="replace"))
    return rc
