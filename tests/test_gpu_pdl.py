"""Programmatic dependent launch inside the captured evaluation graphs: the kernels of a
graph plan are captured with the attribute (counted by hear_pdl_launch_count), and the
result is bit-identical to the same evaluation captured without it (HEAR_PDL=0 in a child
process) and to the oracle."""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_09164_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
from paper_2104_09164_gb300 import hear as H
from paper_2104_09164_gb300.workloads import make_workload
w = make_workload("small")
ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
model = H.hear_model_create(ctx, w.layers, w.clip_dim)
sk, pk, evk = H.hear_keygen(ctx, 301, H.hear_model_rotations(model))
ct = H.hear_encrypt_clips(ctx, pk, w.ct_clips(0), 401, 0)
out = H.hear_evaluate(model, evk, [ct])[0]
np.save(sys.argv[1], H.hear_ciphertext_export(out))
print("pdl", H.hear_pdl_launch_count())
"""


@pytest.fixture(scope="module")
def H():
    from paper_2104_09164_gb300.build import build
    build()
    from paper_2104_09164_gb300 import hear
    return hear


def test_graph_with_and_without_pdl_bit_identical(H, tmp_path):
    if os.environ.get("HEAR_PDL", "1").startswith("0"):
        pytest.skip("PDL switched off in this process")
    w = make_workload("small")
    ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    try:
        model = H.hear_model_create(ctx, w.layers, w.clip_dim)
        steps = H.hear_model_rotations(model)
        sk, pk, evk = H.hear_keygen(ctx, 301, steps)
        ct = H.hear_encrypt_clips(ctx, pk, w.ct_clips(0), 401, 0)
        before = H.hear_pdl_launch_count()
        out = H.hear_evaluate(model, evk, [ct])[0]
        captured = H.hear_pdl_launch_count() - before
        # nearly every kernel of the plan follows another kernel
        assert captured >= 50
        mine = H.hear_ciphertext_export(out)

        path = str(tmp_path / "nopdl.npy")
        env = dict(os.environ, HEAR_PDL="0")
        r = subprocess.run([sys.executable, "-c", CHILD, path], cwd=ROOT, env=env, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        assert "pdl 0" in r.stdout
        assert np.array_equal(np.load(path), mine)

        o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma, threads=os.cpu_count() or 0)
        keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
        z, kk = O.pack_clips(w.ct_clips(0), w.slots)
        x = o.encrypt(keys.pk, z, 401, 0, 2.0 ** w.log2_scale)
        assert np.array_equal(mine, o.to_coeff(o.evaluate(w.layers, x, kk, keys)))
        for h in (ct, out):
            H.hear_ciphertext_destroy(h)
        H.hear_model_destroy(model)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
    finally:
        H.hear_context_destroy(ctx)
