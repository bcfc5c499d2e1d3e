"""CPU-only checks of the C ABI library: it builds, loads, and exports every symbol that
include/hear.h declares (no compute call: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hear.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hear_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2104_09164_gb300.build import build
    return build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    syms = declared_symbols()
    assert len(syms) >= 30
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_the_abi(libpath):
    from paper_2104_09164_gb300 import hear
    names = {n for n in dir(hear) if n.startswith("hear_")}
    missing = [s for s in declared_symbols() if s not in names and s != "hear_last_error"]
    assert not missing, missing


def test_errors_without_gpu_do_not_abort(libpath):
    """Argument errors come back as status codes with a message."""
    from paper_2104_09164_gb300 import hear
    lib = hear.lib
    out = ctypes.c_void_p()
    assert lib.hear_context_create(None, 0, ctypes.byref(out)) == -1
    assert b"null" in lib.hear_last_error()
    assert lib.hear_ciphertext_info(None, None, None, None) == -1


def test_scalar_rounding_is_exact(libpath):
    """hear_dbg_round_scalar (host only) equals round(w q) in exact rational arithmetic, ties
    away from zero -- the rule of the oracle's scalar_residues -- on random, tied, tiny and
    boundary weights, and refuses non-finite or out-of-range ones."""
    from fractions import Fraction
    import numpy as np
    from paper_2104_09164_gb300 import hear

    def exact(w, q):
        f = Fraction(w) * q
        mag = (2 * abs(f.numerator) + f.denominator) // (2 * f.denominator)
        return -mag if f.numerator < 0 else mag

    rng = np.random.default_rng(9)
    qs = [(1 << 40) - 87, (1 << 60) - 93, 1099511480321, 3]
    ws = list(rng.normal(0, 0.3, 200)) + list(rng.normal(0, 1e3, 50)) + [0.0, -0.0, 0.5, -0.5, 1.5, -2.5,
                                                                          2.0 ** -60, -(2.0 ** -70), 5e-324]
    for q in qs:
        for w in ws:
            if abs(Fraction(w) * q) >= 2 ** 62:
                continue
            assert hear.hear_dbg_round_scalar(w, q) == exact(w, q), (w, q)
    # half-integers round away from zero
    assert hear.hear_dbg_round_scalar(0.5, 3) == 2 and hear.hear_dbg_round_scalar(-0.5, 3) == -2
    for bad in (float("nan"), float("inf"), 2.0 ** 30):
        with pytest.raises(hear.HearError):
            hear.hear_dbg_round_scalar(bad, (1 << 40) - 87)


def test_status_codes_match_the_header(libpath):
    from paper_2104_09164_gb300 import hear
    src = open(os.path.join(ROOT, "include", "hear.h")).read()
    for name, val in re.findall(r"#define (HEAR_(?:OK|E_[A-Z]+))\s+\(?(-?\d+)\)?", src):
        assert getattr(hear, name) == int(val), name


def test_params_alpha_is_checked_before_any_device_work(libpath):
    """hear_params_desc.alpha: 0 or n_p is accepted; any other digit size is refused with
    HEAR_E_UNSUPPORTED before the library touches a device"""
    from paper_2104_09164_gb300 import hear
    for alpha in (1, 3):
        with pytest.raises(hear.HearError) as e:
            hear.hear_context_create(14, [60] + [40] * 7, [60, 60], alpha=alpha)
        assert e.value.code == hear.HEAR_E_UNSUPPORTED and "alpha" in str(e.value)
    # a struct with the field in place: the refusal is the alpha check, not a layout error
    assert ctypes.sizeof(hear.hear_params_desc) >= 48


def test_noalloc_refuses_bad_sizes_without_a_gpu(libpath):
    """argument checks of hear_rescale_noalloc that need no device: a null context"""
    from paper_2104_09164_gb300 import hear
    lib = hear.lib
    assert lib.hear_rescale_noalloc(None, None, 0, 1, 2, None, 0, None) == hear.HEAR_E_INVAL
