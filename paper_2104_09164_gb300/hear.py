"""Python binding of the C ABI in include/hear.h (argument marshalling only).

Every function has the name of the C entry point it calls.  All ring arithmetic runs in
the CUDA library ``libhear.so``; if it cannot be loaded the import of this module fails --
there is no CPU fallback.  Handles are opaque integers; release them with the matching
``*_destroy`` call.  ``stream`` arguments accept None (the context's stream), an integer
cudaStream_t, or any object with a ``cuda_stream`` attribute (e.g. ``torch.cuda.Stream``).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhear.so")

HEAR_LAYER_FC = 1
HEAR_LAYER_SQUARE = 2
HEAR_LAYER_FC_SQ_FC = 3
DEFAULT_ROTSUM_RADIX = 8
HEAR_CNN_CONV, HEAR_CNN_QUAD, HEAR_CNN_POOL, HEAR_CNN_GAP, HEAR_CNN_FC = 1, 2, 3, 4, 5
HEAR_CNN_BN_QUAD, HEAR_CNN_AVGPOOL, HEAR_CNN_GAVGPOOL = 6, 7, 8
HEAR_STRATEGY_HYBRID, HEAR_STRATEGY_FULL, HEAR_STRATEGY_BABY, HEAR_STRATEGY_GIANT = 0, 1, 2, 3
HEAR_CNN_OP_DIAG, HEAR_CNN_OP_PACK, HEAR_CNN_OP_ROTSUM, HEAR_CNN_OP_QUAD, HEAR_CNN_OP_BIAS = 1, 2, 3, 4, 5

_vp = ctypes.c_void_p
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i8p = ctypes.POINTER(ctypes.c_int8)
_dp = ctypes.POINTER(ctypes.c_double)
_szp = ctypes.POINTER(ctypes.c_size_t)


class hear_params_desc(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_uint32), ("n_q", ctypes.c_uint32), ("q_bits", _u32p),
                ("n_p", ctypes.c_uint32), ("p_bits", _u32p), ("log2_scale", ctypes.c_double),
                ("sigma", ctypes.c_double), ("alpha", ctypes.c_uint32)]


class hear_layer_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("d_out", ctypes.c_uint32), ("d_in", ctypes.c_uint32),
                ("w", _dp), ("bias", _dp), ("d_out2", ctypes.c_uint32), ("w2", _dp)]


class hear_model_opts(ctypes.Structure):
    _fields_ = [("level", ctypes.c_uint32), ("rotsum_radix", ctypes.c_uint32), ("fc_n1", ctypes.c_uint32),
                ("hoist_moddown", ctypes.c_uint32), ("hoist_sums", ctypes.c_uint32)]


class hear_profile_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class hear_server_config(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("n_slots", ctypes.c_uint32), ("hbm_budget_bytes", ctypes.c_uint64),
                ("staging_cts", ctypes.c_uint32), ("max_pending", ctypes.c_uint32)]


class hear_server_counters(ctypes.Structure):
    _fields_ = [("requests_done", ctypes.c_uint64), ("ciphertexts_done", ctypes.c_uint64),
                ("clips_done", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("pending", ctypes.c_uint64),
                ("max_in_flight_ciphertexts", ctypes.c_uint64), ("bytes_per_ciphertext", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("busy_refusals", ctypes.c_uint64)]


class hear_cnn_input(ctypes.Structure):
    _fields_ = [("conv_dims", ctypes.c_uint32), ("c_in", ctypes.c_uint32), ("h", ctypes.c_uint32),
                ("w", ctypes.c_uint32), ("pitch", ctypes.c_uint32), ("stride", ctypes.c_uint32),
                ("level", ctypes.c_uint32)]


class hear_cnn_layer(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("c_out", ctypes.c_uint32), ("f_h", ctypes.c_uint32),
                ("f_w", ctypes.c_uint32), ("w", _dp), ("bias", _dp), ("a", _dp), ("b", _dp), ("c", _dp),
                ("fast", ctypes.c_uint32), ("strategy", ctypes.c_uint32), ("n1", ctypes.c_uint32),
                ("conv_bias", _dp), ("bn_gamma", _dp), ("bn_beta", _dp), ("bn_mean", _dp), ("bn_var", _dp),
                ("bn_eps", ctypes.c_double), ("act", ctypes.c_double * 3)]


class hear_cnn_op_info(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("layer", ctypes.c_uint32), ("n_in", ctypes.c_uint32),
                ("n_out", ctypes.c_uint32), ("level_in", ctypes.c_uint32), ("level_out", ctypes.c_uint32),
                ("n_babies", ctypes.c_uint32), ("n_giants", ctypes.c_uint32), ("n_keyswitch", ctypes.c_uint32)]


HEAR_OK, HEAR_E_INVAL, HEAR_E_NOMEM, HEAR_E_CUDA, HEAR_E_LEVEL = 0, -1, -2, -3, -4
HEAR_E_SCALE, HEAR_E_NOKEY, HEAR_E_STATE, HEAR_E_FORMAT, HEAR_E_UNSUPPORTED = -5, -6, -7, -8, -9
HEAR_E_TIMEOUT, HEAR_E_BUSY = -10, -11


class HearError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hear error %d: %s" % (code, msg))
        self.code = code


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
# context -> every ctypes callback pair ever installed on it: buffers allocated through a
# hook keep its free function after the hook is replaced, so each pair stays alive until
# the context (and everything made with it) is destroyed
_allocators = {}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libhear.so is not built (run paper_2104_09164_gb300/build.py); "
                          "there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    sig = {
        "hear_last_error": (ctypes.c_char_p, []),
        "hear_context_create": (st, [ctypes.POINTER(hear_params_desc), ctypes.c_int, ctypes.POINTER(_vp)]),
        "hear_context_destroy": (None, [_vp]),
        "hear_set_allocator": (st, [_vp, _ALLOC_FN, _FREE_FN, _vp]),
        "hear_context_primes": (st, [_vp, _u64p, ctypes.c_size_t, _szp]),
        "hear_context_cdt": (st, [_vp, _u64p, ctypes.c_size_t, _szp]),
        "hear_keygen": (st, [_vp, ctypes.c_uint64, _i32p, ctypes.c_size_t, ctypes.POINTER(_vp),
                             ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
        "hear_secret_key_destroy": (None, [_vp]),
        "hear_public_key_destroy": (None, [_vp]),
        "hear_eval_keys_destroy": (None, [_vp]),
        "hear_secret_key_export": (st, [_vp, _i8p, ctypes.c_size_t, _szp]),
        "hear_public_key_export": (st, [_vp, _u64p, ctypes.c_size_t, _szp]),
        "hear_eval_key_export": (st, [_vp, ctypes.c_uint32, _u64p, ctypes.c_size_t, _szp]),
        "hear_encode": (st, [_vp, _dp, ctypes.c_size_t, ctypes.c_double, _i64p, ctypes.c_size_t, _szp]),
        "hear_encrypt": (st, [_vp, _vp, _dp, ctypes.c_size_t, ctypes.c_double, ctypes.c_uint64,
                              ctypes.c_uint64, ctypes.POINTER(_vp), _vp]),
        "hear_encrypt_clips": (st, [_vp, _vp, _dp, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.POINTER(_vp), _vp]),
        "hear_decrypt": (st, [_vp, _vp, _vp, _dp, ctypes.c_size_t, _szp]),
        "hear_ciphertext_destroy": (None, [_vp]),
        "hear_ciphertext_info": (st, [_vp, _u32p, _u32p, _dp]),
        "hear_ciphertext_export": (st, [_vp, _u64p, ctypes.c_size_t, _szp]),
        "hear_ciphertext_import": (st, [_vp, _u64p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_double, ctypes.POINTER(_vp), _vp]),
        "hear_rotate": (st, [_vp, _vp, ctypes.c_int32, ctypes.POINTER(_vp), _vp]),
        "hear_rotate_hoisted": (st, [_vp, _vp, _i32p, ctypes.c_size_t, ctypes.POINTER(_vp), _vp]),
        "hear_rescale": (st, [_vp, ctypes.POINTER(_vp), _vp]),
        "hear_add": (st, [_vp, _vp, ctypes.POINTER(_vp), _vp]),
        "hear_mulplain": (st, [_vp, _dp, ctypes.c_size_t, ctypes.c_double, ctypes.POINTER(_vp), _vp]),
        "hear_multiply_relin": (st, [_vp, _vp, _vp, ctypes.POINTER(_vp), _vp]),
        "hear_model_create": (st, [_vp, ctypes.POINTER(hear_layer_desc), ctypes.c_size_t, ctypes.c_uint32,
                                   ctypes.POINTER(_vp)]),
        "hear_model_destroy": (None, [_vp]),
        "hear_model_create_at_level": (st, [_vp, ctypes.POINTER(hear_layer_desc), ctypes.c_size_t,
                                            ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_vp)]),
        "hear_model_levels": (st, [_vp, _u32p, _u32p]),
        "hear_model_create_ex": (st, [_vp, ctypes.POINTER(hear_layer_desc), ctypes.c_size_t, ctypes.c_uint32,
                                      ctypes.POINTER(hear_model_opts), ctypes.POINTER(_vp)]),
        "hear_ciphertext_drop_level": (st, [_vp, ctypes.c_uint32, ctypes.POINTER(_vp), _vp]),
        "hear_model_rotations": (st, [_vp, _i32p, ctypes.c_size_t, _szp]),
        "hear_model_output_positions": (st, [_vp, _u32p, ctypes.c_size_t, _szp]),
        "hear_evaluate": (st, [_vp, _vp, ctypes.POINTER(_vp), ctypes.c_size_t, ctypes.POINTER(_vp), _vp]),
        "hear_evaluate_layer": (st, [_vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp), ctypes.c_size_t,
                                     ctypes.POINTER(_vp), _vp]),
        "hear_evaluate_host": (st, [_vp, _vp, _u64p, ctypes.c_size_t, ctypes.c_double, _u64p, ctypes.c_size_t,
                                    _szp, _u32p, _dp, _vp]),
        "hear_multi_create": (st, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_size_t, _u32p, _dp,
                                   ctypes.POINTER(_vp)]),
        "hear_multi_evaluate": (st, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp]),
        "hear_multi_destroy": (None, [_vp]),
        "hear_server_create": (st, [_vp, _vp, ctypes.POINTER(hear_server_config), ctypes.POINTER(_vp)]),
        "hear_server_submit": (st, [_vp, _u64p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_double,
                                    ctypes.POINTER(ctypes.c_uint64)]),
        "hear_server_poll": (st, [_vp, ctypes.c_uint64, _u64p, ctypes.c_size_t, _szp, ctypes.POINTER(ctypes.c_int)]),
        "hear_server_stats": (st, [_vp, ctypes.POINTER(hear_server_counters)]),
        "hear_server_wait": (st, [_vp, ctypes.c_uint64, ctypes.c_uint32, _u64p, ctypes.c_size_t, _szp]),
        "hear_server_pause": (st, [_vp, ctypes.c_int]),
        "hear_server_destroy": (None, [_vp]),
        "hear_cnn_collapse": (st, [ctypes.POINTER(hear_cnn_input), ctypes.POINTER(hear_cnn_layer), ctypes.c_size_t,
                                   _dp, ctypes.c_size_t, _szp]),
        "hear_cnn_create": (st, [_vp, ctypes.POINTER(hear_cnn_input), ctypes.POINTER(hear_cnn_layer),
                                 ctypes.c_size_t, ctypes.POINTER(_vp)]),
        "hear_cnn_destroy": (None, [_vp]),
        "hear_cnn_rotations": (st, [_vp, _i32p, ctypes.c_size_t, _szp]),
        "hear_cnn_ops": (st, [_vp, ctypes.POINTER(hear_cnn_op_info), ctypes.c_size_t, _szp]),
        "hear_cnn_output_slots": (st, [_vp, _u32p, ctypes.c_size_t, _szp]),
        "hear_cnn_encrypt": (st, [_vp, _vp, _vp, _dp, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(_vp),
                                  _vp]),
        "hear_cnn_evaluate": (st, [_vp, _vp, ctypes.c_size_t, ctypes.c_size_t, ctypes.POINTER(_vp),
                                   ctypes.c_size_t, ctypes.POINTER(_vp), _vp]),
        "hear_simd_model_create": (st, [_vp, ctypes.POINTER(hear_layer_desc), ctypes.c_size_t, ctypes.c_uint32,
                                        ctypes.POINTER(_vp)]),
        "hear_simd_model_info": (st, [_vp, _u32p, _u32p, _u32p, _u32p]),
        "hear_simd_model_destroy": (None, [_vp]),
        "hear_simd_encrypt": (st, [_vp, _vp, _dp, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_double,
                                   ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(_vp), _vp]),
        "hear_simd_batch_info": (st, [_vp, _u32p, _u32p, _dp]),
        "hear_simd_batch_export": (st, [_vp, _u64p, ctypes.c_size_t, _szp]),
        "hear_simd_batch_import": (st, [_vp, _u64p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_double,
                                        ctypes.POINTER(_vp), _vp]),
        "hear_simd_batch_destroy": (None, [_vp]),
        "hear_simd_evaluate": (st, [_vp, _vp, _vp, ctypes.POINTER(_vp), _vp]),
        "hear_simd_evaluate_host": (st, [_vp, _vp, _u64p, ctypes.c_double, _u64p, ctypes.c_size_t, _szp, _u32p,
                                         _dp, _vp]),
        "hear_simd_decrypt": (st, [_vp, _vp, _vp, ctypes.c_size_t, _dp, ctypes.c_size_t, _szp]),
        "hear_rescale_noalloc": (st, [_vp, _u64p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint32, _u64p,
                                      ctypes.c_size_t, _vp]),
        "hear_profile_begin": (st, [_vp]),
        "hear_profile_end": (st, [_vp, ctypes.POINTER(hear_profile_entry), ctypes.c_size_t, _szp]),
        "hear_launch_count": (ctypes.c_uint64, []),
        "hear_pdl_launch_count": (ctypes.c_uint64, []),
        "hear_ntt_tune": (st, [_vp, ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8),
                               ctypes.POINTER(ctypes.c_float)]),
        "hear_ntt_set_variant": (st, [_vp, ctypes.c_int]),
        "hear_ks_tune": (st, [_vp, ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8),
                              ctypes.POINTER(ctypes.c_float)]),
        "hear_ks_get_table": (st, [_vp, ctypes.POINTER(ctypes.c_uint8)]),
        "hear_ks_set_table": (st, [_vp, ctypes.POINTER(ctypes.c_uint8)]),
        "hear_ks_set_variant": (st, [_vp, ctypes.c_int]),
        "hear_ntt_get_table": (st, [_vp, ctypes.POINTER(ctypes.c_uint8)]),
        "hear_ntt_set_table": (st, [_vp, ctypes.POINTER(ctypes.c_uint8)]),
        "hear_dbg_imad_peak": (st, [_vp, ctypes.c_int, ctypes.c_uint32, _dp]),
        "hear_dbg_bfly_peak": (st, [_vp, ctypes.c_int, ctypes.c_uint32, _dp]),
        "hear_async_status": (st, [_vp, ctypes.POINTER(ctypes.c_uint32)]),
        "hear_dbg_wait_probe": (st, [_vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_uint32)]),
        "hear_dbg_round_scalar": (st, [ctypes.c_double, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64)]),
        "hear_dbg_poly_mul": (st, [_vp, ctypes.c_uint32, _u64p, _u64p, _u64p]),
        "hear_dbg_ntt_roundtrip": (st, [_vp, _u64p, ctypes.c_size_t]),
        "hear_dbg_ntt_time": (st, [_vp, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                   ctypes.POINTER(ctypes.c_float)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _check(rc):
    if rc != 0:
        raise HearError(rc, lib.hear_last_error().decode(errors="replace"))


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return _vp(s.cuda_stream)
    return _vp(int(s))


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a, t):
    return a.ctypes.data_as(t)


# ---------------------------------------------------------------- context
def hear_context_create(log_n, q_bits, p_bits, log2_scale=40.0, sigma=3.2, device=0, alpha=0):
    qb = _arr(q_bits, np.uint32)
    pb = _arr(p_bits, np.uint32)
    d = hear_params_desc(log_n, len(qb), _p(qb, _u32p), len(pb), _p(pb, _u32p), float(log2_scale), float(sigma),
                         int(alpha))
    h = _vp()
    _check(lib.hear_context_create(ctypes.byref(d), int(device), ctypes.byref(h)))
    return h.value


def hear_context_destroy(ctx):
    lib.hear_context_destroy(ctx)
    _allocators.pop(ctx, None)   # released only after the library has freed everything


def _vec_out(fn, handle, dtype, ptr_t, *pre):
    n = ctypes.c_size_t(0)
    fn(handle, *pre, None, 0, ctypes.byref(n))
    out = np.empty(n.value, dtype=dtype)
    _check(fn(handle, *pre, _p(out, ptr_t), n.value, ctypes.byref(n)))
    return out


def hear_set_allocator(ctx, alloc, free):
    """alloc(bytes, stream) -> device pointer (int, 0 on failure), free(ptr, stream); both
    None = back to the stream-ordered pool.  Streams are passed as integers (0 = none)."""
    a = _ALLOC_FN(lambda n, st, u: alloc(int(n), int(st or 0)) or None) if alloc is not None else _ALLOC_FN()
    f = _FREE_FN(lambda p, st, u: free(int(p), int(st or 0))) if free is not None else _FREE_FN()
    _check(lib.hear_set_allocator(ctx, a, f, None))
    if alloc is not None:
        _allocators.setdefault(ctx, []).append((a, f))


def hear_context_primes(ctx):
    return [int(x) for x in _vec_out(lib.hear_context_primes, ctx, np.uint64, _u64p)]


def hear_context_cdt(ctx):
    return [int(x) for x in _vec_out(lib.hear_context_cdt, ctx, np.uint64, _u64p)]


# ---------------------------------------------------------------- keys
def hear_keygen(ctx, seed, rot_steps=()):
    steps = _arr(list(rot_steps), np.int32)
    sk, pk, evk = _vp(), _vp(), _vp()
    _check(lib.hear_keygen(ctx, int(seed), _p(steps, _i32p) if len(steps) else None, len(steps),
                           ctypes.byref(sk), ctypes.byref(pk), ctypes.byref(evk)))
    return sk.value, pk.value, evk.value


def hear_secret_key_destroy(h):
    lib.hear_secret_key_destroy(h)


def hear_public_key_destroy(h):
    lib.hear_public_key_destroy(h)


def hear_eval_keys_destroy(h):
    lib.hear_eval_keys_destroy(h)


def hear_secret_key_export(sk):
    return _vec_out(lib.hear_secret_key_export, sk, np.int8, _i8p)


def hear_public_key_export(pk):
    return _vec_out(lib.hear_public_key_export, pk, np.uint64, _u64p)


def hear_eval_key_export(evk, galois):
    return _vec_out(lib.hear_eval_key_export, evk, np.uint64, _u64p, ctypes.c_uint32(galois))


# ---------------------------------------------------------------- encoding / encryption
def hear_encode(ctx, z, scale):
    z = _arr(z, np.float64)
    n = ctypes.c_size_t(0)
    out = np.empty(2 * len(z), dtype=np.int64)
    _check(lib.hear_encode(ctx, _p(z, _dp), len(z), float(scale), _p(out, _i64p), len(out), ctypes.byref(n)))
    return out


def hear_encrypt(ctx, pk, z, scale, seed, ct_id, stream=None):
    z = _arr(z, np.float64)
    h = _vp()
    _check(lib.hear_encrypt(ctx, pk, _p(z, _dp), len(z), float(scale), int(seed), int(ct_id), ctypes.byref(h),
                            _stream(stream)))
    return h.value


def hear_encrypt_clips(ctx, pk, clips, seed, ct_id, stream=None):
    c = _arr(np.atleast_2d(clips), np.float64)
    h = _vp()
    _check(lib.hear_encrypt_clips(ctx, pk, _p(c, _dp), c.shape[0], c.shape[1], int(seed), int(ct_id),
                                  ctypes.byref(h), _stream(stream)))
    return h.value


def hear_decrypt(ctx, sk, ct):
    n = ctypes.c_size_t(0)
    lib.hear_decrypt(ctx, sk, ct, None, 0, ctypes.byref(n))
    out = np.empty(n.value, dtype=np.float64)
    _check(lib.hear_decrypt(ctx, sk, ct, _p(out, _dp), n.value, ctypes.byref(n)))
    return out


def hear_ciphertext_destroy(ct):
    lib.hear_ciphertext_destroy(ct)


def hear_ciphertext_info(ct):
    lv, npl, sc = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_double()
    _check(lib.hear_ciphertext_info(ct, ctypes.byref(lv), ctypes.byref(npl), ctypes.byref(sc)))
    return lv.value, npl.value, sc.value


def hear_ciphertext_export(ct):
    lv, npl, _ = hear_ciphertext_info(ct)
    flat = _vec_out(lib.hear_ciphertext_export, ct, np.uint64, _u64p)
    return flat.reshape(npl, lv + 1, -1)


def hear_ciphertext_import(ctx, words, level, n_poly, scale, stream=None):
    w = _arr(words, np.uint64).reshape(-1)
    h = _vp()
    _check(lib.hear_ciphertext_import(ctx, _p(w, _u64p), w.size, int(level), int(n_poly), float(scale),
                                      ctypes.byref(h), _stream(stream)))
    return h.value


# ---------------------------------------------------------------- primitive operations
def hear_rotate(evk, ct, step, stream=None):
    h = _vp()
    _check(lib.hear_rotate(evk, ct, int(step), ctypes.byref(h), _stream(stream)))
    return h.value


def hear_rotate_hoisted(evk, ct, steps, stream=None):
    s = _arr(list(steps), np.int32)
    outs = (_vp * len(s))()
    _check(lib.hear_rotate_hoisted(evk, ct, _p(s, _i32p), len(s), outs, _stream(stream)))
    return [o for o in outs]


def hear_rescale(ct, stream=None):
    h = _vp()
    _check(lib.hear_rescale(ct, ctypes.byref(h), _stream(stream)))
    return h.value


def hear_add(a, b, stream=None):
    h = _vp()
    _check(lib.hear_add(a, b, ctypes.byref(h), _stream(stream)))
    return h.value


def hear_mulplain(ct, z, pt_scale, stream=None):
    z = _arr(z, np.float64)
    h = _vp()
    _check(lib.hear_mulplain(ct, _p(z, _dp), len(z), float(pt_scale), ctypes.byref(h), _stream(stream)))
    return h.value


def hear_multiply_relin(evk, a, b, stream=None):
    h = _vp()
    _check(lib.hear_multiply_relin(evk, a, b, ctypes.byref(h), _stream(stream)))
    return h.value


# ---------------------------------------------------------------- network
def _layer_descs(layers):
    """-> (hear_layer_desc array, the arrays it points into)"""
    descs = (hear_layer_desc * len(layers))()
    keep = []
    for i, layer in enumerate(layers):
        d = descs[i]
        if layer[0] == "fc":
            W = _arr(layer[1], np.float64)
            keep.append(W)
            d.kind, d.d_out, d.d_in, d.w = HEAR_LAYER_FC, W.shape[0], W.shape[1], _p(W, _dp)
            if len(layer) > 2 and layer[2] is not None:
                b = _arr(layer[2], np.float64).reshape(-1)
                if b.size != W.shape[0]:
                    raise ValueError("FC bias needs d_out values")
                keep.append(b)
                d.bias = _p(b, _dp)
        elif layer[0] == "square":
            d.kind = HEAR_LAYER_SQUARE
        elif layer[0] == "fc_sq_fc":
            W1, W2 = _arr(layer[1], np.float64), _arr(layer[2], np.float64)
            keep += [W1, W2]
            d.kind, d.d_out, d.d_in, d.w = HEAR_LAYER_FC_SQ_FC, W1.shape[0], W1.shape[1], _p(W1, _dp)
            d.d_out2, d.w2 = W2.shape[0], _p(W2, _dp)
        else:
            raise ValueError(layer[0])
    return descs, keep


def hear_model_create(ctx, layers, clip_dim, level=None, rotsum_radix=None, fc_n1=None, hoist_moddown=False,
                      hoist_sums=False):
    """layers: sequence of ("fc", W[, bias]) | ("square",) | ("fc_sq_fc", W1, W2) with float64 matrices;
    level: input level (None = the top level); rotsum_radix, fc_n1, hoist_moddown, hoist_sums:
    see hear_model_opts"""
    descs, keep = _layer_descs(layers)
    h = _vp()
    if rotsum_radix is not None or fc_n1 is not None or hoist_moddown or hoist_sums:
        opts = hear_model_opts(int(level or 0), int(rotsum_radix or 0), int(fc_n1 or 0), int(bool(hoist_moddown)),
                               int(bool(hoist_sums)))
        _check(lib.hear_model_create_ex(ctx, descs, len(layers), int(clip_dim), ctypes.byref(opts), ctypes.byref(h)))
    elif level is None:
        _check(lib.hear_model_create(ctx, descs, len(layers), int(clip_dim), ctypes.byref(h)))
    else:
        _check(lib.hear_model_create_at_level(ctx, descs, len(layers), int(clip_dim), int(level), ctypes.byref(h)))
    return h.value


def hear_model_create_ex(ctx, layers, clip_dim, level=0, rotsum_radix=0):
    return hear_model_create(ctx, layers, clip_dim, level or None, rotsum_radix or DEFAULT_ROTSUM_RADIX)


def hear_model_create_at_level(ctx, layers, clip_dim, level):
    return hear_model_create(ctx, layers, clip_dim, level)


def hear_model_levels(m):
    a, b = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib.hear_model_levels(m, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def hear_ciphertext_drop_level(ct, level, stream=None):
    h = _vp()
    _check(lib.hear_ciphertext_drop_level(ct, int(level), ctypes.byref(h), _stream(stream)))
    return h.value


def hear_model_destroy(m):
    lib.hear_model_destroy(m)


def hear_model_rotations(m):
    return [int(x) for x in _vec_out(lib.hear_model_rotations, m, np.int32, _i32p)]


def hear_model_output_positions(m):
    return [int(x) for x in _vec_out(lib.hear_model_output_positions, m, np.uint32, _u32p)]


def hear_evaluate(m, evk, cts, stream=None):
    ins = (_vp * len(cts))(*cts)
    outs = (_vp * len(cts))()
    _check(lib.hear_evaluate(m, evk, ins, len(cts), outs, _stream(stream)))
    return [o for o in outs]


def hear_evaluate_layer(m, layer, evk, cts, stream=None):
    ins = (_vp * len(cts))(*cts)
    outs = (_vp * len(cts))()
    _check(lib.hear_evaluate_layer(m, int(layer), evk, ins, len(cts), outs, _stream(stream)))
    return [o for o in outs]


def hear_evaluate_host(m, evk, in_words, n_ct, scale, out=None, stream=None):
    w = _arr(in_words, np.uint64).reshape(-1)
    n = ctypes.c_size_t(0)
    lv, sc = ctypes.c_uint32(), ctypes.c_double()
    if out is None:
        lib.hear_evaluate_host(m, evk, _p(w, _u64p), int(n_ct), float(scale), None, 0, ctypes.byref(n),
                               None, None, None)
        out = np.empty(n.value, dtype=np.uint64)
    _check(lib.hear_evaluate_host(m, evk, _p(w, _u64p), int(n_ct), float(scale), _p(out, _u64p), out.size,
                                  ctypes.byref(n), ctypes.byref(lv), ctypes.byref(sc), _stream(stream)))
    return out, lv.value, sc.value


# ---------------------------------------------------------------- several networks, one launch
def hear_multi_create(models, evks, n_ct, scales):
    """one CUDA-graph launch evaluating job i = (models[i], evks[i]) on n_ct[i] ciphertexts"""
    J = len(models)
    m = (_vp * J)(*models)
    k = (_vp * J)(*evks)
    n = np.ascontiguousarray(n_ct, dtype=np.uint32)
    s = np.ascontiguousarray(scales, dtype=np.float64)
    h = _vp()
    _check(lib.hear_multi_create(m, k, J, _p(n, _u32p), _p(s, _dp), ctypes.byref(h)))
    return h.value


def hear_multi_evaluate(mu, cts, stream=None):
    """cts: the jobs' inputs concatenated -> their results in the same order"""
    ins = (_vp * len(cts))(*cts)
    outs = (_vp * len(cts))()
    _check(lib.hear_multi_evaluate(mu, ins, outs, _stream(stream)))
    return [o for o in outs]


def hear_multi_destroy(mu):
    lib.hear_multi_destroy(mu)


# ---------------------------------------------------------------- slot-batched evaluation
def hear_simd_model_create(ctx, layers, level=0):
    """layers as for hear_model_create; level 0 = the top level"""
    descs, keep = _layer_descs(layers)
    h = _vp()
    _check(lib.hear_simd_model_create(ctx, descs, len(layers), int(level), ctypes.byref(h)))
    return h.value


def hear_simd_model_info(m):
    """-> (d_in, d_out, level_in, level_out)"""
    v = [ctypes.c_uint32() for _ in range(4)]
    _check(lib.hear_simd_model_info(m, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def hear_simd_model_destroy(m):
    lib.hear_simd_model_destroy(m)


def hear_simd_encrypt(ctx, pk, x, seed, level=0, scale=0.0, stream=None):
    """x: [n_clips][n_features] -> batch of n_features ciphertexts, clip c in slot c"""
    a = _arr(np.atleast_2d(x), np.float64)
    h = _vp()
    _check(lib.hear_simd_encrypt(ctx, pk, _p(a, _dp), a.shape[0], a.shape[1], float(scale), int(seed), int(level),
                                 ctypes.byref(h), _stream(stream)))
    return h.value


def hear_simd_batch_info(b):
    """-> (n_ct, level, scale)"""
    n, lv, sc = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_double()
    _check(lib.hear_simd_batch_info(b, ctypes.byref(n), ctypes.byref(lv), ctypes.byref(sc)))
    return n.value, lv.value, sc.value


def hear_simd_batch_export(b):
    n_ct, lv, _ = hear_simd_batch_info(b)
    return _vec_out(lib.hear_simd_batch_export, b, np.uint64, _u64p).reshape(n_ct, 2, lv + 1, -1)


def hear_simd_batch_import(ctx, words, n_ct, level, scale, stream=None):
    w = _arr(words, np.uint64).reshape(-1)
    h = _vp()
    _check(lib.hear_simd_batch_import(ctx, _p(w, _u64p), int(n_ct), int(level), float(scale), ctypes.byref(h),
                                      _stream(stream)))
    return h.value


def hear_simd_batch_destroy(b):
    lib.hear_simd_batch_destroy(b)


def hear_simd_evaluate(m, evk, batch, stream=None):
    h = _vp()
    _check(lib.hear_simd_evaluate(m, evk, batch, ctypes.byref(h), _stream(stream)))
    return h.value


def hear_simd_evaluate_host(m, evk, in_words, scale, out=None, stream=None):
    w = _arr(in_words, np.uint64).reshape(-1)
    n = ctypes.c_size_t(0)
    lv, sc = ctypes.c_uint32(), ctypes.c_double()
    if out is None:
        lib.hear_simd_evaluate_host(m, evk, _p(w, _u64p), float(scale), None, 0, ctypes.byref(n), None, None, None)
        out = np.empty(n.value, dtype=np.uint64)
    _check(lib.hear_simd_evaluate_host(m, evk, _p(w, _u64p), float(scale), _p(out, _u64p), out.size,
                                       ctypes.byref(n), ctypes.byref(lv), ctypes.byref(sc), _stream(stream)))
    return out, lv.value, sc.value


def hear_simd_decrypt(ctx, sk, batch, n_clips):
    """-> [n_clips][n_ct]"""
    n_ct = hear_simd_batch_info(batch)[0]
    out = np.empty(int(n_clips) * n_ct, dtype=np.float64)
    n = ctypes.c_size_t(0)
    _check(lib.hear_simd_decrypt(ctx, sk, batch, int(n_clips), _p(out, _dp), out.size, ctypes.byref(n)))
    return out.reshape(int(n_clips), n_ct)


# ---------------------------------------------------------------- skeleton CNN
_STRATEGIES = {"hybrid": HEAR_STRATEGY_HYBRID, "full": HEAR_STRATEGY_FULL, "baby": HEAR_STRATEGY_BABY,
               "giant": HEAR_STRATEGY_GIANT}


def _strategy(s):
    """"full" | "baby" | "giant" | ("hybrid", n1) | None (hybrid, default n1) -> (code, n1)"""
    if s is None:
        return HEAR_STRATEGY_HYBRID, 0
    if isinstance(s, str):
        return _STRATEGIES[s], 0
    return _STRATEGIES[s[0]], int(s[1])


def hear_cnn_create(ctx, spec, strategies=None):
    """spec: network dict {"conv_dims", "c_in", "h", "w", ["pitch", "stride"],
    "layers": [("conv", W[c_out][c_in][fh][fw], fast) | ("bn_quad", conv_bias, gamma, beta,
    mean, var, eps, (a, b, c)) | ("avgpool",) | ("gavgpool",) | ("quad", A, B, C) | ("pool",) |
    ("gap",) | ("fc", W, bias)]}: as trained (the library collapses bn_quad / avgpool /
    gavgpool) or already collapsed; strategies: one per conv / fc layer (see _strategy)"""
    inp, descs, keep = _cnn_descs(spec, strategies)
    h = _vp()
    _check(lib.hear_cnn_create(ctx, ctypes.byref(inp), descs, len(descs), ctypes.byref(h)))
    return h.value


def hear_cnn_collapse(spec):
    """host only: the collapsed network's doubles in layer order (CONV weights, QUAD A, B, C,
    FC weights) as the library computes them"""
    inp, descs, keep = _cnn_descs(spec, None)
    n = ctypes.c_size_t(0)
    lib.hear_cnn_collapse(ctypes.byref(inp), descs, len(descs), None, 0, ctypes.byref(n))
    out = np.empty(n.value, dtype=np.float64)
    _check(lib.hear_cnn_collapse(ctypes.byref(inp), descs, len(descs), _p(out, _dp), out.size, ctypes.byref(n)))
    return out


def _cnn_descs(spec, strategies):
    inp = hear_cnn_input(int(spec["conv_dims"]), int(spec["c_in"]), int(spec["h"]), int(spec["w"]),
                         int(spec.get("pitch", 0)), int(spec.get("stride", 1)), int(spec.get("level", 0)))
    layers = spec["layers"]
    descs = (hear_cnn_layer * len(layers))()
    keep = []
    si = 0
    for i, layer in enumerate(layers):
        d = descs[i]
        kind = layer[0]
        if kind == "conv":
            W = _arr(layer[1], np.float64)
            keep.append(W)
            d.kind, d.c_out, d.f_h, d.f_w, d.w = HEAR_CNN_CONV, W.shape[0], W.shape[2], W.shape[3], _p(W, _dp)
            d.fast = 1 if layer[2] else 0
            d.strategy, d.n1 = _strategy(None if strategies is None else strategies[si])
            si += 1
        elif kind == "quad":
            a, b, c = (_arr(v, np.float64) for v in layer[1:4])
            keep += [a, b, c]
            d.kind, d.a, d.b, d.c = HEAR_CNN_QUAD, _p(a, _dp), _p(b, _dp), _p(c, _dp)
        elif kind == "bn_quad":
            bias, gamma, beta, mean, var = (None if v is None else _arr(v, np.float64) for v in layer[1:6])
            keep += [v for v in (bias, gamma, beta, mean, var) if v is not None]
            d.kind = HEAR_CNN_BN_QUAD
            d.conv_bias = _p(bias, _dp) if bias is not None else None
            d.bn_gamma, d.bn_beta, d.bn_mean, d.bn_var = (_p(v, _dp) for v in (gamma, beta, mean, var))
            d.bn_eps = float(layer[6])
            for i, v in enumerate(layer[7]):
                d.act[i] = float(v)
        elif kind in ("pool", "avgpool"):
            d.kind = HEAR_CNN_POOL if kind == "pool" else HEAR_CNN_AVGPOOL
        elif kind in ("gap", "gavgpool"):
            d.kind = HEAR_CNN_GAP if kind == "gap" else HEAR_CNN_GAVGPOOL
        elif kind == "fc":
            W = _arr(layer[1], np.float64)
            keep.append(W)
            d.kind, d.c_out, d.w = HEAR_CNN_FC, W.shape[0], _p(W, _dp)
            if len(layer) > 2 and layer[2] is not None:
                bias = _arr(layer[2], np.float64)
                keep.append(bias)
                d.bias = _p(bias, _dp)
            d.strategy, d.n1 = _strategy(None if strategies is None else strategies[si])
            si += 1
        else:
            raise ValueError(kind)
    return inp, descs, keep


def hear_cnn_destroy(m):
    lib.hear_cnn_destroy(m)


def hear_cnn_rotations(m):
    return [int(x) for x in _vec_out(lib.hear_cnn_rotations, m, np.int32, _i32p)]


def hear_cnn_ops(m):
    n = ctypes.c_size_t(0)
    lib.hear_cnn_ops(m, None, 0, ctypes.byref(n))
    arr = (hear_cnn_op_info * n.value)()
    _check(lib.hear_cnn_ops(m, arr, n.value, ctypes.byref(n)))
    return [{f: getattr(a, f) for f, _ in hear_cnn_op_info._fields_} for a in arr]


def hear_cnn_output_slots(m):
    return [int(x) for x in _vec_out(lib.hear_cnn_output_slots, m, np.uint32, _u32p)]


def hear_cnn_encrypt(ctx, pk, m, x, seed, ct_id, stream=None):
    """x: float64[c_in][h][w] -> the input ciphertexts of one sample"""
    xx = _arr(x, np.float64).reshape(-1)
    n_in = hear_cnn_ops(m)[0]["n_in"]
    outs = (_vp * n_in)()
    _check(lib.hear_cnn_encrypt(ctx, pk, m, _p(xx, _dp), int(seed), int(ct_id), outs, _stream(stream)))
    return [o for o in outs]


def hear_cnn_evaluate(m, evk, op0, op1, cts, n_samples, stream=None):
    """cts: n_samples * n_in handles (sample-major) -> n_samples * n_out handles"""
    ops = hear_cnn_ops(m)
    n_out = ops[op1 - 1]["n_out"]
    ins = (_vp * len(cts))(*cts)
    outs = (_vp * (n_out * n_samples))()
    _check(lib.hear_cnn_evaluate(m, evk, int(op0), int(op1), ins, int(n_samples), outs, _stream(stream)))
    return [o for o in outs]


# ---------------------------------------------------------------- serving
def hear_server_create(m, evk, max_batch=32, n_slots=2, hbm_budget_bytes=64 << 30, staging_cts=0, max_pending=0):
    cfg = hear_server_config(int(max_batch), int(n_slots), int(hbm_budget_bytes), int(staging_cts), int(max_pending))
    h = _vp()
    _check(lib.hear_server_create(m, evk, ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def hear_server_submit(s, words, n_ct, n_clips, scale):
    w = _arr(words, np.uint64).reshape(-1)
    rid = ctypes.c_uint64()
    _check(lib.hear_server_submit(s, _p(w, _u64p), int(n_ct), int(n_clips), float(scale), ctypes.byref(rid)))
    return rid.value


def hear_server_poll(s, request_id, out_words):
    """-> result array (uint64, out_words words) once done, else None"""
    out = np.empty(int(out_words), dtype=np.uint64)
    n = ctypes.c_size_t(0)
    done = ctypes.c_int(0)
    _check(lib.hear_server_poll(s, int(request_id), _p(out, _u64p), out.size, ctypes.byref(n), ctypes.byref(done)))
    return out[:n.value] if done.value else None


def hear_server_wait(s, request_id, out_words, timeout_ms=1000):
    """-> result array once done (blocks up to timeout_ms; HearError HEAR_E_TIMEOUT after)"""
    out = np.empty(int(out_words), dtype=np.uint64)
    n = ctypes.c_size_t(0)
    _check(lib.hear_server_wait(s, int(request_id), int(timeout_ms), _p(out, _u64p), out.size, ctypes.byref(n)))
    return out[:n.value]


def hear_server_pause(s, paused=True):
    _check(lib.hear_server_pause(s, 1 if paused else 0))


def hear_server_stats(s):
    st = hear_server_counters()
    _check(lib.hear_server_stats(s, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in hear_server_counters._fields_}


def hear_server_destroy(s):
    lib.hear_server_destroy(s)


def hear_rescale_noalloc(ctx, words, level, n_poly, stream=None, n=None):
    """rescale from/to host arrays (coefficient domain) without device allocation; n = the
    ring size N (default: from words.size); the library checks words.size itself"""
    w = _arr(words, np.uint64).reshape(-1)
    if n is None:
        n = max(1, w.size // (n_poly * (level + 1)))
    out = np.empty(n_poly * max(level, 0) * n, dtype=np.uint64)
    _check(lib.hear_rescale_noalloc(ctx, _p(w, _u64p), w.size, int(level), int(n_poly), _p(out, _u64p), out.size,
                                    _stream(stream)))
    return out.reshape(n_poly, level, n)


# ---------------------------------------------------------------- tracing
def hear_profile_begin(ctx):
    _check(lib.hear_profile_begin(ctx))


def hear_profile_end(ctx):
    """-> {stage: (launches, total_ms, algorithmic_bytes)}"""
    n = ctypes.c_size_t(0)
    buf = (hear_profile_entry * 256)()
    _check(lib.hear_profile_end(ctx, buf, 256, ctypes.byref(n)))
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms), float(buf[i].bytes))
            for i in range(n.value)}


def hear_launch_count():
    return int(lib.hear_launch_count())


def hear_pdl_launch_count():
    return int(lib.hear_pdl_launch_count())


# ---------------------------------------------------------------- debug
def hear_dbg_round_scalar(w, q):
    """round(w q) exactly, ties away from zero (host only)"""
    v = ctypes.c_int64()
    _check(lib.hear_dbg_round_scalar(float(w), int(q), ctypes.byref(v)))
    return v.value


def hear_dbg_imad_peak(ctx, kind=0, iters=4096):
    """lane operations per second of mad.wide.u32 (kind 0) or mad.lo.u32 (kind 1)"""
    v = ctypes.c_double()
    _check(lib.hear_dbg_imad_peak(ctx, int(kind), int(iters), ctypes.byref(v)))
    return v.value


def hear_dbg_bfly_peak(ctx, inverse=False, iters=2048):
    """butterflies per second of the NTT arithmetic on register-resident radix-16 units"""
    v = ctypes.c_double()
    _check(lib.hear_dbg_bfly_peak(ctx, 1 if inverse else 0, int(iters), ctypes.byref(v)))
    return v.value


HEAR_NTT_WIDE, HEAR_NTT_NARROW, HEAR_NTT_FUSED, HEAR_NTT_TINY = 0, 1, 2, 3


def hear_ntt_tune(ctx, max_limbs=512, iters=5):
    """time the NTT launch variants; returns (choice uint8[2][16], ms float32[2][16][4])"""
    choice = np.zeros((2, 16), dtype=np.uint8)
    ms = np.zeros((2, 16, 4), dtype=np.float32)
    _check(lib.hear_ntt_tune(ctx, int(max_limbs), int(iters), _p(choice, ctypes.POINTER(ctypes.c_uint8)),
                             _p(ms, ctypes.POINTER(ctypes.c_float))))
    return choice, ms


def hear_ntt_get_table(ctx):
    """-> the variant table as a 32-character string (forward buckets, then inverse)"""
    t = np.zeros(32, dtype=np.uint8)
    _check(lib.hear_ntt_get_table(ctx, _p(t, ctypes.POINTER(ctypes.c_uint8))))
    return "".join(str(int(x)) for x in t)


def hear_ntt_set_table(ctx, table):
    t = np.array([int(ch) for ch in table], dtype=np.uint8)
    _check(lib.hear_ntt_set_table(ctx, _p(t, ctypes.POINTER(ctypes.c_uint8))))


def hear_ks_tune(ctx, max_ct=32, iters=5):
    """time the key-switch / inner-sum launch forms; returns (choice uint8[3][8], ms float32[3][8][8])"""
    choice = np.zeros((3, 8), dtype=np.uint8)
    ms = np.zeros((3, 8, 8), dtype=np.float32)
    _check(lib.hear_ks_tune(ctx, int(max_ct), int(iters), _p(choice, ctypes.POINTER(ctypes.c_uint8)),
                            _p(ms, ctypes.POINTER(ctypes.c_float))))
    return choice, ms


def hear_ks_get_table(ctx):
    """-> the form table as a 24-character string (inner products, shared-digit products, inner sums)"""
    t = np.zeros(24, dtype=np.uint8)
    _check(lib.hear_ks_get_table(ctx, _p(t, ctypes.POINTER(ctypes.c_uint8))))
    return "".join(str(int(x)) for x in t)


def hear_ks_set_table(ctx, table):
    t = np.array([int(ch) for ch in table], dtype=np.uint8)
    _check(lib.hear_ks_set_table(ctx, _p(t, ctypes.POINTER(ctypes.c_uint8))))


def hear_ks_set_variant(ctx, variant):
    _check(lib.hear_ks_set_variant(ctx, int(variant)))


def hear_async_status(ctx):
    """-> bounded device waits that ran out since the last check (0 = none); the C call
    returns HEAR_E_TIMEOUT when some did, reported here as the count"""
    n = ctypes.c_uint32()
    s = lib.hear_async_status(ctx, ctypes.byref(n))
    if s not in (0, HEAR_E_TIMEOUT):
        _check(s)
    return int(n.value)


def hear_dbg_wait_probe(ctx, limit_cycles):
    """one bounded wait on an mbarrier nothing completes: True if it ran out"""
    v = ctypes.c_uint32()
    _check(lib.hear_dbg_wait_probe(ctx, int(limit_cycles), ctypes.byref(v)))
    return bool(v.value)


def hear_ntt_set_variant(ctx, variant):
    _check(lib.hear_ntt_set_variant(ctx, int(variant)))


def hear_dbg_poly_mul(ctx, prime, a, b):
    a, b = _arr(a, np.uint64), _arr(b, np.uint64)
    out = np.empty_like(a)
    _check(lib.hear_dbg_poly_mul(ctx, int(prime), _p(a, _u64p), _p(b, _u64p), _p(out, _u64p)))
    return out


def hear_dbg_ntt_roundtrip(ctx, limbs):
    """limbs: [n_limb][N]; limb i uses prime i mod (n_q + n_p)"""
    x = _arr(limbs, np.uint64).copy()
    _check(lib.hear_dbg_ntt_roundtrip(ctx, _p(x, _u64p), x.shape[0]))
    return x


def hear_dbg_ntt_time(ctx, n_limb, iters=20):
    """-> (ms per forward NTT, ms per inverse NTT) over n_limb limbs"""
    f, i = ctypes.c_float(), ctypes.c_float()
    _check(lib.hear_dbg_ntt_time(ctx, int(n_limb), int(iters), ctypes.byref(f), ctypes.byref(i)))
    return f.value, i.value
