"""CPU oracle for the RNS-CKKS hot path of HEAR / Fast-HEAR (arXiv 2104.09164).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference legs may import this module.  It shares no code with the CUDA
library: the ring arithmetic lives in the plain-C ``hear_oracle.c`` (loaded through
ctypes) and the composition below follows the paper step by step:

* encrypted matrix-vector product in diagonal form, re-associated baby-step/giant-step
  with the identity rho^(a+b) = rho^a o rho^b (Methods, "Algorithmic and cryptographic
  optimizations", giant-step / baby-step strategies): baby rotations rho^(i) of the
  input, plaintexts pre-rotated by rho^(-j*n1), giant rotations rho^(j*n1) of the
  partial sums;
* hoisting (same paragraph, item (i)): the baby rotations share one ModUp;
* lazy rescaling (item (ii)): products are summed, then rescaled once;
* level-aware encoding (item (iii)): each weight plaintext only carries the limbs of the
  level at which it is used;
* FC layer (Methods, "Non-convolutional layers"), polynomial activation x^2, and the
  collapse of adjacent layers into one polynomial evaluation (same paragraph);
* data encryption with interlaced copies (Methods, "Data encryption");
* slot-batched evaluation of the same FC / x^2 networks (one clip per slot, one
  ciphertext per feature): the FC layer of Methods "Non-convolutional layers" becomes a
  sum of ciphertexts times plaintext scalars, each scalar the encoding of a constant slot
  vector (the canonical embedding maps a constant polynomial c to c in every slot), with
  one lazy rescale per output and no rotation.

Ciphertexts here are numpy uint64 arrays [n_poly][level+1][N] in the oracle's own NTT
domain; ``to_coeff`` gives the coefficient domain used for every comparison.
"""
import ctypes
import math
import os
from fractions import Fraction
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .build import build_oracle

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i8p = ctypes.POINTER(ctypes.c_int8)
_dp = ctypes.POINTER(ctypes.c_double)

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = ctypes.CDLL(path)
        sig = {
            "or_mulmod": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]),
            "or_is_prime": (ctypes.c_int, [ctypes.c_uint64]),
            "or_gen_primes": (ctypes.c_int, [ctypes.c_uint32, _u32p, ctypes.c_uint32, _u64p]),
            "or_ctx_create": (ctypes.c_void_p, [ctypes.c_uint32, ctypes.c_uint32, _u32p,
                                                ctypes.c_uint32, _u32p, ctypes.c_double]),
            "or_ctx_destroy": (None, [ctypes.c_void_p]),
            "or_ctx_primes": (ctypes.c_int, [ctypes.c_void_p, _u64p]),
            "or_ctx_psi": (ctypes.c_int, [ctypes.c_void_p, _u64p]),
            "or_set_threads": (ctypes.c_int, [ctypes.c_int]),
            "or_ntt_fwd": (ctypes.c_int, [ctypes.c_void_p, _u32p, ctypes.c_uint32, _u64p]),
            "or_ntt_inv": (ctypes.c_int, [ctypes.c_void_p, _u32p, ctypes.c_uint32, _u64p]),
            "or_chacha20_block": (None, [_u32p, ctypes.c_uint32, _u32p, _u32p]),
            "or_stream_words": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_size_t, _u64p]),
            "or_cdt_table": (ctypes.c_int, [ctypes.c_void_p, _u64p, ctypes.c_uint32, _u32p]),
            "or_sample_ternary": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                         ctypes.c_size_t, _i8p]),
            "or_sample_gauss": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                               ctypes.c_uint64, ctypes.c_size_t, _i8p]),
            "or_sample_uniform": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_size_t, _u64p]),
            "or_encode": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.c_double, _i64p,
                                         ctypes.POINTER(ctypes.c_int)]),
            "or_dd_cossin": (None, [ctypes.c_uint64, ctypes.c_uint64, _dp, _dp, _dp, _dp]),
            "or_keygen_sk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, _i8p]),
            "or_sk_ntt": (ctypes.c_int, [ctypes.c_void_p, _i8p, _u64p]),
            "or_keygen_pk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, _i8p, _u64p]),
            "or_keygen_swk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, _i8p,
                                             ctypes.c_uint32, _u64p]),
            "or_dnum": (ctypes.c_uint32, [ctypes.c_void_p, ctypes.c_uint32]),
            "or_encrypt": (ctypes.c_int, [ctypes.c_void_p, _u64p, _i64p, ctypes.c_uint64,
                                          ctypes.c_uint64, _u64p]),
            "or_decrypt": (ctypes.c_int, [ctypes.c_void_p, _u64p, ctypes.c_uint32, _u64p, _u64p]),
            "or_to_coeff": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                           _u64p, _u64p]),
            "or_from_coeff": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                             _u64p, _u64p]),
            "or_encode_pt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _i64p, _u64p]),
            "or_mul_ext": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p, _u64p]),
            "or_add_ext": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p, _u64p]),
            "or_scale_p_ext": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p]),
            "or_encode_pt_ext": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _i64p, _u64p]),
            "or_add": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                      _u64p, _u64p, _u64p]),
            "or_mulplain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _u64p, _u64p, _u64p]),
            "or_tensor": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _u64p, _u64p, _u64p]),
            "or_automorphism_coeff": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _u32p,
                                                     ctypes.c_uint32, _u64p, _u64p]),
            "or_automorphism_ntt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32,
                                                   ctypes.c_uint32, _u64p, _u64p]),
            "or_modup": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _u64p, _u64p]),
            "or_ks_inner": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _u64p, _u64p,
                                           ctypes.c_uint32, _u64p]),
            "or_moddown": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _u64p, _u64p]),
            "or_rescale": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                          _u64p, _u64p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def P(a, t=_u64p):
    return a.ctypes.data_as(t)


def _chk(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed (%d)" % (what, rc))


# purpose ids of the randomness streams (must match the C side's enum)
P_SK, P_PK_A, P_PK_E, P_KSK_A, P_KSK_E, P_ENC_V, P_ENC_E0, P_ENC_E1 = 1, 2, 3, 4, 5, 8, 9, 10


class Ct:
    """A ciphertext: data [n_poly][level+1][N] (oracle NTT domain), level, scale."""

    def __init__(self, data, level, scale):
        self.data = np.ascontiguousarray(data, dtype=np.uint64)
        self.level = level
        self.scale = float(scale)

    @property
    def n_poly(self):
        return self.data.shape[0]


class Keys:
    def __init__(self):
        self.s = None        # int8 [N] ternary secret
        self.s_ntt = None    # [n_q+n_p][N]
        self.pk = None       # [2][n_q][N]
        self.relin = None    # [dnum][2][n_q+n_p][N]
        self.rot = {}        # galois -> [dnum][2][n_q+n_p][N]


# copies folded per rotate-and-sum round (radix - 1 rotations sharing one ModUp); 2 = the
# plain log2-depth tree; 8 is the evaluation's default
ROTSUM_RADIX = 8


def galois_for_step(step: int, n: int) -> int:
    """rho^step (left rotation by step slots) <-> X -> X^(5^step mod 2N)"""
    return pow(5, step % (n // 2), 2 * n)


def bsgs_split(D: int):
    """n1 = smallest power of two with n1^2 >= D (at most D), n2 = ceil(D / n1)."""
    n1 = 1
    while n1 * n1 < D:
        n1 *= 2
    n1 = min(n1, D)
    return n1, (D + n1 - 1) // n1


class Oracle:
    def __init__(self, log_n, q_bits, p_bits, sigma=3.2, threads=0):
        L = lib()
        if threads:
            L.or_set_threads(threads)
        self.log_n, self.n = log_n, 1 << log_n
        self.n_q, self.n_p = len(q_bits), len(p_bits)
        qb = np.array(q_bits, dtype=np.uint32)
        pb = np.array(p_bits, dtype=np.uint32)
        self.h = L.or_ctx_create(log_n, self.n_q, P(qb, _u32p), self.n_p, P(pb, _u32p), sigma)
        if not self.h:
            raise RuntimeError("oracle context creation failed")
        pr = np.zeros(self.n_q + self.n_p, dtype=np.uint64)
        L.or_ctx_primes(self.h, P(pr))
        self.primes = [int(x) for x in pr]
        self.q = self.primes[:self.n_q]
        self.p = self.primes[self.n_q:]
        self.L = self.n_q - 1

    def __del__(self):
        try:
            if self.h:
                lib().or_ctx_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # ---------------- helpers ----------------
    def dnum(self, level):
        return lib().or_dnum(self.h, level)

    def ntt_fwd(self, a, prime_idx):
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        pi = np.ascontiguousarray(prime_idx, dtype=np.uint32)
        _chk(lib().or_ntt_fwd(self.h, P(pi, _u32p), len(pi), P(a)), "ntt_fwd")
        return a

    def ntt_inv(self, a, prime_idx):
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        pi = np.ascontiguousarray(prime_idx, dtype=np.uint32)
        _chk(lib().or_ntt_inv(self.h, P(pi, _u32p), len(pi), P(a)), "ntt_inv")
        return a

    def to_coeff(self, ct: Ct):
        out = np.empty_like(ct.data)
        _chk(lib().or_to_coeff(self.h, ct.level, ct.n_poly, P(ct.data), P(out)), "to_coeff")
        return out

    def from_coeff(self, data, level, scale):
        data = np.ascontiguousarray(data, dtype=np.uint64)
        out = np.empty_like(data)
        _chk(lib().or_from_coeff(self.h, level, data.shape[0], P(data), P(out)), "from_coeff")
        return Ct(out, level, scale)

    # ---------------- encoding ----------------
    def encode(self, z, scale):
        """round(scale * tau^-1(z)) for N/2 real slot values z"""
        z = np.ascontiguousarray(z, dtype=np.float64)
        assert z.shape == (self.n // 2,)
        m = np.empty(self.n, dtype=np.int64)
        ties = ctypes.c_int(0)
        _chk(lib().or_encode(self.h, P(z, _dp), float(scale), P(m, _i64p), ctypes.byref(ties)),
             "encode")
        return m, ties.value

    def encode_pt(self, z, scale, level):
        m, ties = self.encode(z, scale)
        if ties:
            raise RuntimeError("encoding hit %d near-ties" % ties)
        pt = np.empty((level + 1, self.n), dtype=np.uint64)
        _chk(lib().or_encode_pt(self.h, level, P(m, _i64p), P(pt)), "encode_pt")
        return pt

    def decode(self, coeffs_centered, scale):
        """slot values z_j = sum_k (m_k / scale) zeta^(5^j k), zeta = e^(i pi / N)"""
        n = self.n
        v = np.asarray([float(x) for x in coeffs_centered], dtype=np.float64) / scale
        F = np.fft.ifft(np.concatenate([v, np.zeros(n)])) * (2 * n)
        t = np.array([pow(5, j, 2 * n) for j in range(n // 2)], dtype=np.int64)
        return F[t].real

    # ---------------- keys ----------------
    def keygen(self, seed, galois_list=(), relin=True):
        L = lib()
        k = Keys()
        k.s = np.empty(self.n, dtype=np.int8)
        _chk(L.or_keygen_sk(self.h, seed, P(k.s, _i8p)), "keygen_sk")
        k.s_ntt = np.empty((self.n_q + self.n_p, self.n), dtype=np.uint64)
        _chk(L.or_sk_ntt(self.h, P(k.s, _i8p), P(k.s_ntt)), "sk_ntt")
        k.pk = np.empty((2, self.n_q, self.n), dtype=np.uint64)
        _chk(L.or_keygen_pk(self.h, seed, P(k.s, _i8p), P(k.pk)), "keygen_pk")
        if relin:
            k.relin = self.switching_key(seed, k.s, 1)
        for g in galois_list:
            k.rot[int(g)] = self.switching_key(seed, k.s, int(g))
        return k

    def switching_key(self, seed, s, galois):
        out = np.empty((self.dnum(self.L), 2, self.n_q + self.n_p, self.n), dtype=np.uint64)
        _chk(lib().or_keygen_swk(self.h, seed, P(s, _i8p), galois, P(out)), "keygen_swk")
        return out

    # ---------------- encryption ----------------
    def encrypt_m(self, pk, m, seed, ct_id, scale):
        ct = np.empty((2, self.n_q, self.n), dtype=np.uint64)
        m = np.ascontiguousarray(m, dtype=np.int64)
        _chk(lib().or_encrypt(self.h, P(pk), P(m, _i64p), seed, ct_id, P(ct)), "encrypt")
        return Ct(ct, self.L, scale)

    def encrypt(self, pk, z, seed, ct_id, scale):
        m, ties = self.encode(z, scale)
        if ties:
            raise RuntimeError("encoding hit %d near-ties" % ties)
        return self.encrypt_m(pk, m, seed, ct_id, scale)

    def decrypt_residues(self, keys, ct: Ct):
        out = np.empty((ct.level + 1, self.n), dtype=np.uint64)
        _chk(lib().or_decrypt(self.h, P(keys.s_ntt), ct.level, P(ct.data), P(out)), "decrypt")
        return out

    def crt_centered(self, residues, level):
        """CRT with Python integers to [0, Q_l), then centred into (-Q_l/2, Q_l/2]."""
        qs = self.q[:level + 1]
        Q = 1
        for q in qs:
            Q *= q
        acc = np.zeros(self.n, dtype=object)
        for i, q in enumerate(qs):
            qh = Q // q
            inv = pow(qh % q, -1, q)
            y = (residues[i].astype(object) * inv) % q
            acc = acc + y * qh
        acc = acc % Q
        half = Q // 2
        return [int(x) - Q if int(x) > half else int(x) for x in acc]

    def decrypt(self, keys, ct: Ct):
        r = self.decrypt_residues(keys, ct)
        return self.decode(self.crt_centered(r, ct.level), ct.scale)

    # ---------------- primitives ----------------
    def add(self, a: Ct, b: Ct):
        assert a.level == b.level and a.n_poly == b.n_poly
        out = np.empty_like(a.data)
        _chk(lib().or_add(self.h, a.level, a.n_poly, P(a.data), P(b.data), P(out)), "add")
        return Ct(out, a.level, a.scale)

    def add_plain(self, ct: Ct, pt):
        """ct + pt: the plaintext (same level, NTT domain) is added to c0; scale unchanged"""
        pt = np.ascontiguousarray(pt, dtype=np.uint64)
        assert pt.shape == (ct.level + 1, self.n)
        out = ct.data.copy()
        c0 = np.empty((1, ct.level + 1, self.n), dtype=np.uint64)
        _chk(lib().or_add(self.h, ct.level, 1, P(np.ascontiguousarray(ct.data[:1])), P(pt), P(c0)), "add")
        out[0] = c0[0]
        return Ct(out, ct.level, ct.scale)

    def drop_level(self, ct: Ct):
        """the same ciphertext over Q_(level-1): the last residue is discarded (no division,
        scale unchanged), which is how a ciphertext meets a partner one level down"""
        return Ct(np.ascontiguousarray(ct.data[:, :ct.level]), ct.level - 1, ct.scale)

    def mulplain(self, ct: Ct, pt, pt_scale):
        out = np.empty_like(ct.data)
        pt = np.ascontiguousarray(pt, dtype=np.uint64)
        _chk(lib().or_mulplain(self.h, ct.level, P(ct.data), P(pt), P(out)), "mulplain")
        return Ct(out, ct.level, ct.scale * pt_scale)

    def tensor(self, a: Ct, b: Ct):
        out = np.empty((3, a.level + 1, self.n), dtype=np.uint64)
        _chk(lib().or_tensor(self.h, a.level, P(a.data), P(b.data), P(out)), "tensor")
        return Ct(out, a.level, a.scale * b.scale)

    def modup(self, level, d):
        W = level + 1 + self.n_p
        ext = np.empty((self.dnum(level), W, self.n), dtype=np.uint64)
        d = np.ascontiguousarray(d, dtype=np.uint64)
        _chk(lib().or_modup(self.h, level, P(d), P(ext)), "modup")
        return ext

    def ks_inner(self, level, ext, swk, galois):
        W = level + 1 + self.n_p
        out = np.empty((2, W, self.n), dtype=np.uint64)
        _chk(lib().or_ks_inner(self.h, level, P(ext), P(swk), galois, P(out)), "ks_inner")
        return out

    def moddown(self, level, x):
        out = np.empty((level + 1, self.n), dtype=np.uint64)
        x = np.ascontiguousarray(x, dtype=np.uint64)
        _chk(lib().or_moddown(self.h, level, P(x), P(out)), "moddown")
        return out

    def automorphism(self, level, n_poly, data, galois):
        out = np.empty_like(data)
        for p in range(n_poly):
            src = np.ascontiguousarray(data[p])
            dst = np.empty_like(src)
            _chk(lib().or_automorphism_ntt(self.h, level + 1, galois, P(src), P(dst)), "auto")
            out[p] = dst
        return out

    def rescale(self, ct: Ct):
        out = np.empty((ct.n_poly, ct.level, self.n), dtype=np.uint64)
        _chk(lib().or_rescale(self.h, ct.level, ct.n_poly, P(ct.data), P(out)), "rescale")
        return Ct(out, ct.level - 1, ct.scale / float(self.q[ct.level]))

    def keyswitch(self, level, d, swk, galois=1):
        """hybrid key switching of d (ModUp -> inner product -> ModDown); returns (u0, u1)"""
        ext = self.modup(level, d)
        inner = self.ks_inner(level, ext, swk, galois)
        return self.moddown(level, inner[0]), self.moddown(level, inner[1])

    def rotate_hoisted(self, ct: Ct, steps, keys: Keys):
        """rho^step(ct) for several steps sharing one ModUp of c1; sigma_g is applied to the
        extended digits (hoisting)."""
        ext = self.modup(ct.level, ct.data[1])
        outs = []
        for st in steps:
            g = galois_for_step(st, self.n)
            inner = self.ks_inner(ct.level, ext, keys.rot[g], g)
            u0 = self.moddown(ct.level, inner[0])
            u1 = self.moddown(ct.level, inner[1])
            c0g = self.automorphism(ct.level, 1, ct.data[:1], g)[0]
            out = np.empty_like(ct.data)
            out[0] = self.add(Ct(c0g[None], ct.level, 1), Ct(u0[None], ct.level, 1)).data[0]
            out[1] = u1
            outs.append(Ct(out, ct.level, ct.scale))
        return outs

    # ---------------- hoisted ModDown (baby steps kept over Q_l u P) ----------------
    def encode_pt_ext(self, z, scale, level):
        m, ties = self.encode(z, scale)
        if ties:
            raise RuntimeError("encoding hit %d near-ties" % ties)
        W = level + 1 + self.n_p
        pt = np.empty((W, self.n), dtype=np.uint64)
        _chk(lib().or_encode_pt_ext(self.h, level, P(m, _i64p), P(pt)), "encode_pt_ext")
        return pt

    def mul_ext(self, level, a, pt):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.empty_like(a)
        _chk(lib().or_mul_ext(self.h, level, a.shape[0], P(a), P(np.ascontiguousarray(pt)), P(out)), "mul_ext")
        return out

    def add_ext(self, level, a, b):
        out = np.empty_like(a)
        _chk(lib().or_add_ext(self.h, level, a.shape[0], P(np.ascontiguousarray(a)), P(np.ascontiguousarray(b)),
                              P(out)), "add_ext")
        return out

    def scale_p_ext(self, ct: Ct):
        W = ct.level + 1 + self.n_p
        out = np.empty((ct.n_poly, W, self.n), dtype=np.uint64)
        _chk(lib().or_scale_p_ext(self.h, ct.level, ct.n_poly, P(np.ascontiguousarray(ct.data)), P(out)),
             "scale_p_ext")
        return out

    def rotate_hoisted_ext(self, ct: Ct, steps, keys: Keys):
        """rho^step(ct) before ModDown, over Q_l u P: (P sigma_g(c0) + u0, u1) with (u0, u1)
        the key inner product of the hoisted ModUp of c1 (one ModUp for all steps)"""
        ext = self.modup(ct.level, ct.data[1])
        outs = []
        for st in steps:
            g = galois_for_step(st, self.n)
            inner = self.ks_inner(ct.level, ext, keys.rot[g], g)
            c0g = self.automorphism(ct.level, 1, ct.data[:1], g)
            pc0 = self.scale_p_ext(Ct(c0g, ct.level, 1))
            out = inner.copy()
            out[:1] = self.add_ext(ct.level, inner[:1], pc0)
            outs.append(out)
        return outs

    def rotate(self, ct: Ct, step, keys: Keys):
        return self.rotate_hoisted(ct, [step], keys)[0]

    def relinearize(self, ct3: Ct, keys: Keys):
        u0, u1 = self.keyswitch(ct3.level, ct3.data[2], keys.relin, 1)
        out = np.empty((2, ct3.level + 1, self.n), dtype=np.uint64)
        out[0] = self.add(Ct(ct3.data[:1], ct3.level, 1), Ct(u0[None], ct3.level, 1)).data[0]
        out[1] = self.add(Ct(ct3.data[1:2], ct3.level, 1), Ct(u1[None], ct3.level, 1)).data[0]
        return Ct(out, ct3.level, ct3.scale)

    def mul_relin_rescale(self, a: Ct, b: Ct, keys: Keys):
        """ciphertext product: tensor, relinearise, then rescale"""
        return self.rescale(self.relinearize(self.tensor(a, b), keys))

    # ---------------- linear algebra on slots ----------------
    @staticmethod
    def diag_vector(W, i, M):
        """i-th generalized diagonal in the pos space of size M:
        diag_i[p] = W[p mod d_out][(p + i) mod d_in]"""
        d_out, d_in = W.shape
        p = np.arange(M)
        return W[p % d_out, (p + i) % d_in]

    @staticmethod
    def expand(v, k):
        """pos-space vector of size M -> N/2 slots, slot p*k + c holds v[p]"""
        return np.repeat(np.asarray(v, dtype=np.float64), k)

    def fc(self, ct: Ct, W, k, keys: Keys, pool=None, radix=ROTSUM_RADIX, n1=None, dh=False, hs=False, bias=None):
        """Encrypted FC layer, BSGS diagonal form with hoisted baby steps and one lazy
        rescale, followed by rotate-and-sum; output replicated with period d_out.
        n1: baby steps (default bsgs_split); dh: hoisted ModDown -- the baby rotations stay
        over Q_l u P (P-scaled identity as baby 0), the inner sums are formed there with
        plaintexts over Q_l u P and each giant-step sum is ModDowned once.
        hs: hoisted sums -- the giant rotations of the inner sums j >= 1 are kept over
        Q_l u P as (P sigma(c0) + u0, u1), added to inner sum 0 over Q_l u P (P-scaled when it
        is over Q_l) and ModDowned once, and so is every rotate-and-sum round (rotsum).
        bias (d_out values): added after the rotate-and-sum as the plaintext b[p mod d_out] in
        every slot p*k + c, encoded at the output's scale and level."""
        d_out, d_in = W.shape
        M = (self.n // 2) // k
        assert d_in <= M and M % d_in == 0 and d_in % d_out == 0
        D = d_out
        if n1 is None:
            n1, n2 = bsgs_split(D)
        else:
            n1 = min(n1, D)
            n2 = (D + n1 - 1) // n1
        level = ct.level
        ql = float(self.q[level])
        steps = [b * k for b in range(1, n1)]
        if dh:
            babies = [self.scale_p_ext(ct)] + (self.rotate_hoisted_ext(ct, steps, keys) if n1 > 1 else [])
        else:
            babies = [ct] + (self.rotate_hoisted(ct, steps, keys) if n1 > 1 else [])
        enc = self.encode_pt_ext if dh else self.encode_pt

        def pt_for(j, b):
            v = np.roll(self.diag_vector(W, j * n1 + b, M), j * n1)   # rho^(-j n1)
            return enc(self.expand(v, k), ql, level)

        jobs = [(j, b) for j in range(n2) for b in range(n1) if j * n1 + b < D]
        if pool is None:
            pool = ThreadPoolExecutor(max_workers=os.cpu_count() or 4)
        pts = dict(zip(jobs, pool.map(lambda jb: pt_for(*jb), jobs)))
        acc = None
        acc_ext = None
        for j in range(n2):
            inner = None
            for b in range(n1):
                if j * n1 + b >= D:
                    break
                if dh:
                    prod = self.mul_ext(level, babies[b], pts[(j, b)])
                    inner = prod if inner is None else self.add_ext(level, inner, prod)
                else:
                    prod = self.mulplain(babies[b], pts[(j, b)], ql)
                    inner = prod if inner is None else self.add(inner, prod)
            if hs and j == 0:
                # the sum over Q_l u P starts with inner sum 0 (P-scaled when over Q_l)
                acc_ext = inner if dh else self.scale_p_ext(inner)
                continue
            if dh:
                data = np.stack([self.moddown(level, inner[p]) for p in range(2)])
                inner = Ct(data, level, ct.scale * ql)
            if hs:
                rot = self.rotate_hoisted_ext(inner, [j * n1 * k], keys)[0]
                acc_ext = self.add_ext(level, acc_ext, rot)
                continue
            if j > 0:
                inner = self.rotate(inner, j * n1 * k, keys)
            acc = inner if acc is None else self.add(acc, inner)
        if hs:
            acc = Ct(np.stack([self.moddown(level, acc_ext[p]) for p in range(2)]), level, ct.scale * ql)
        out = self.rescale(acc)
        out = self.rotsum(out, d_out, d_in // d_out, k, keys, radix, hs)
        if bias is not None:
            b = np.asarray(bias, dtype=np.float64)[np.arange(M) % d_out]
            out = self.add_plain(out, self.encode_pt(self.expand(b, k), out.scale, out.level))
        return out

    def rotsum(self, ct: Ct, step, count, k, keys: Keys, radix, hs=False):
        """sum of the count (a power of two) copies rho^(j*step*k)(ct), j < count, folded in
        rounds of up to radix - 1 hoisted rotations: out <- out + sum_j rho^(j*s*k)(out),
        s <- s*r (radix 2 is the plain rotate-and-sum tree).  hs: each round is summed over
        Q_l u P -- P out + sum_j (P sigma_j(c0) + u0_j, u1_j) -- and ModDowned once."""
        while count > 1:
            r = min(radix, count)
            steps = [j * step * k for j in range(1, r)]
            if hs:
                acc = self.scale_p_ext(ct)
                for x in self.rotate_hoisted_ext(ct, steps, keys):
                    acc = self.add_ext(ct.level, acc, x)
                ct = Ct(np.stack([self.moddown(ct.level, acc[p]) for p in range(2)]), ct.level, ct.scale)
            else:
                for x in self.rotate_hoisted(ct, steps, keys):
                    ct = self.add(ct, x)
            step *= r
            count //= r
        return ct

    def square(self, ct: Ct, keys: Keys):
        return self.mul_relin_rescale(ct, ct, keys)

    def fc_sq_fc(self, ct: Ct, W1, W2, k, keys: Keys, pool=None, radix=ROTSUM_RADIX, hs=False):
        """Collapsed FC -> x^2 -> FC: out_c = sum_r W2[c,r] y_r^2 with y = W1 x, as the
        product of y and u = U x, U[(c, r), :] = W2[c, r] W1[r, :], both at one level,
        then rotate-and-sum over r.  Logit c lands at pos c * d1."""
        d1 = W1.shape[0]
        d2 = W2.shape[0]
        U = (W2[:, :, None] * W1[None, :, :]).reshape(d2 * d1, W1.shape[1])
        y = self.fc(ct, W1, k, keys, pool, radix, hs=hs)
        u = self.fc(ct, U, k, keys, pool, radix, hs=hs)
        z = self.mul_relin_rescale(y, u, keys)
        return self.rotsum(z, 1, d1, k, keys, radix, hs)

    def evaluate(self, layers, ct: Ct, k, keys: Keys, pool=None, radix=ROTSUM_RADIX, n1=None, dh=False, hs=False):
        for layer in layers:
            if layer[0] == "fc":
                ct = self.fc(ct, layer[1], k, keys, pool, radix, n1, dh, hs, layer[2] if len(layer) > 2 else None)
            elif layer[0] == "square":
                ct = self.square(ct, keys)
            elif layer[0] == "fc_sq_fc":
                ct = self.fc_sq_fc(ct, layer[1], layer[2], k, keys, pool, radix, hs)
            else:
                raise ValueError(layer[0])
        return ct

    # ---------------- slot-batched evaluation (one clip per slot) ----------------
    def scalar_residues(self, w, level):
        """The plaintext scalar for weight w at scale q_level: the constant slot vector w
        encodes to the constant polynomial round(w q_level), rounded exactly with ties away
        from zero like the encoder, i.e. one residue per limb t <= level.
        w: float array of any shape -> uint64 [..., level+1]."""
        w = np.asarray(w, dtype=np.float64)
        ql = self.q[level]
        c = []
        for v in w.ravel():
            f = Fraction(float(v)) * ql
            mag = (2 * abs(f.numerator) + f.denominator) // (2 * f.denominator)
            c.append(-mag if f.numerator < 0 else mag)
        out = np.empty((len(c), level + 1), dtype=np.uint64)
        for t in range(level + 1):
            qt = self.q[t]
            out[:, t] = [x % qt for x in c]
        return out.reshape(w.shape + (level + 1,))

    def mul_scalar(self, ct: Ct, res, pt_scale):
        """ct times the constant polynomial with residues res[t]: in the NTT domain every
        evaluation of limb t is multiplied by res[t]"""
        pt = np.repeat(np.asarray(res, dtype=np.uint64)[:ct.level + 1, None], self.n, axis=1)
        return self.mulplain(ct, pt, pt_scale)

    def encrypt_simd(self, pk, X, seed, scale):
        """Clips X [n_clips][d] (n_clips <= N/2) -> d ciphertexts; ciphertext i encrypts
        the slot vector (X[0][i], .., X[n_clips-1][i], 0, ..) with randomness stream i"""
        X = np.asarray(X, dtype=np.float64)
        assert X.shape[0] <= self.n // 2
        out = []
        for i in range(X.shape[1]):
            z = np.zeros(self.n // 2)
            z[:X.shape[0]] = X[:, i]
            out.append(self.encrypt(pk, z, seed, i, scale))
        return out

    def fc_simd(self, cts, W):
        """FC layer with one clip per slot: y_o = rescale(sum_i [W[o,i]]_{q_l} x_i), the
        scalars at scale q_l (lazy rescaling: the products are summed, then rescaled once)"""
        W = np.asarray(W, dtype=np.float64)
        d_out, d_in = W.shape
        assert len(cts) == d_in
        level = cts[0].level
        R = self.scalar_residues(W, level)
        ql = float(self.q[level])
        out = []
        for o in range(d_out):
            acc = self.mul_scalar(cts[0], R[o, 0], ql)
            for i in range(1, d_in):
                acc = self.add(acc, self.mul_scalar(cts[i], R[o, i], ql))
            out.append(self.rescale(acc))
        return out

    def fc_sq_fc_simd(self, cts, W1, W2, keys: Keys):
        """Collapsed FC -> x^2 -> FC with one clip per slot: out_c = sum_r W2[c,r] y_r^2,
        y = W1 x, as sum_r y_r * u_(c,r) with u_(c,r) = U[(c,r)] x, U[(c,r), :] =
        W2[c, r] W1[r, :] (both FC outputs one level down), the degree-2 products summed
        over r before one relinearisation and one rescale per output"""
        W1 = np.asarray(W1, dtype=np.float64)
        W2 = np.asarray(W2, dtype=np.float64)
        d1, d2 = W1.shape[0], W2.shape[0]
        U = (W2[:, :, None] * W1[None, :, :]).reshape(d2 * d1, W1.shape[1])
        y = self.fc_simd(cts, W1)
        u = self.fc_simd(cts, U)
        out = []
        for c in range(d2):
            t = self.tensor(y[0], u[c * d1])
            for r in range(1, d1):
                t = self.add(t, self.tensor(y[r], u[c * d1 + r]))
            out.append(self.rescale(self.relinearize(t, keys)))
        return out

    def evaluate_simd(self, layers, cts, keys: Keys):
        for layer in layers:
            if layer[0] == "fc":
                if len(layer) > 2 and layer[2] is not None:
                    raise ValueError("the slot-batched form has no FC bias")
                cts = self.fc_simd(cts, layer[1])
            elif layer[0] == "square":
                cts = [self.square(c, keys) for c in cts]
            elif layer[0] == "fc_sq_fc":
                cts = self.fc_sq_fc_simd(cts, layer[1], layer[2], keys)
            else:
                raise ValueError(layer[0])
        return cts

    def decrypt_simd(self, keys, cts, n_clips):
        """-> [n_clips][len(cts)]: slot c of ciphertext o is output o of clip c"""
        return np.stack([self.decrypt(keys, ct)[:n_clips] for ct in cts], axis=1)


def rotsum_steps(step, count, radix):
    """rotation amounts (pos units) of Oracle.rotsum"""
    out = []
    while count > 1:
        r = min(radix, count)
        out += [j * step for j in range(1, r)]
        step *= r
        count //= r
    return out


def rotation_steps(layers, clip_dim, k, radix=ROTSUM_RADIX, n1_opt=None):
    """pos-space rotation amounts (times k = slots) every key switch of the network needs"""
    steps = set()

    def fc_steps(d_out, d_in):
        if n1_opt is None:
            n1, n2 = bsgs_split(d_out)
        else:
            n1 = min(n1_opt, d_out)
            n2 = (d_out + n1 - 1) // n1
        for b in range(1, n1):
            steps.add(b * k)
        for j in range(1, n2):
            steps.add(j * n1 * k)
        steps.update(s * k for s in rotsum_steps(d_out, d_in // d_out, radix))

    for layer in layers:
        if layer[0] == "fc":
            fc_steps(*layer[1].shape)
        elif layer[0] == "fc_sq_fc":
            W1, W2 = layer[1], layer[2]
            fc_steps(*W1.shape)
            fc_steps(W2.shape[0] * W1.shape[0], W1.shape[1])
            steps.update(s * k for s in rotsum_steps(1, W1.shape[0], radix))
    return sorted(steps)


def pack_clips(clips, slots):
    """Interlaced packing: k = slots / clip_dim lanes, slot p*k + c holds clip (c mod n)[p]."""
    clips = np.atleast_2d(np.asarray(clips, dtype=np.float64))
    n, d = clips.shape
    k = slots // d
    assert k * d == slots and 1 <= n <= k
    z = np.empty(slots)
    for c in range(k):
        z[c::k] = clips[c % n]
    return z, k


def output_positions(layers):
    """pos of logit c in the decrypted pos space"""
    last = layers[-1]
    if last[0] == "fc":
        return list(range(last[1].shape[0]))
    if last[0] == "fc_sq_fc":
        d1 = last[1].shape[0]
        return [c * d1 for c in range(last[2].shape[0])]
    raise ValueError(last[0])
