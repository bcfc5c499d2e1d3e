"""Several networks in one CUDA-graph launch (hear_multi_*): the small network (N = 2^14) and
the large one (N = 2^15) evaluated as concurrent branches of one graph give the same
ciphertexts, bit for bit, as separate evaluations (themselves bit-exact against the
oracle), and logits within 2^-15 of FP64; inputs at the wrong level are refused."""
import numpy as np
import pytest

from paper_2104_09164_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2104_09164_gb300.build import build
    build()
    from paper_2104_09164_gb300 import hear
    return hear


class Job:
    def __init__(self, H, name, n_clips):
        self.H, self.w = H, make_workload(name, n_clips)
        w = self.w
        self.ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
        self.model = H.hear_model_create(self.ctx, w.layers, w.clip_dim)
        self.sk, self.pk, self.evk = H.hear_keygen(self.ctx, 301, H.hear_model_rotations(self.model))
        self.cts = [H.hear_encrypt_clips(self.ctx, self.pk, w.ct_clips(i), 401, i) for i in range(w.n_ct)]

    def logits(self, outs):
        H, w = self.H, self.w
        k = w.slots // w.clip_dim
        pos = H.hear_model_output_positions(self.model)
        got = []
        for i, o in enumerate(outs):
            dec = H.hear_decrypt(self.ctx, self.sk, o)
            for c in range(min(w.clips_per_ct, w.n_clips - i * w.clips_per_ct)):
                got.append([dec[p * k + c] for p in pos])
        return np.array(got)

    def close(self):
        H = self.H
        for c in self.cts:
            H.hear_ciphertext_destroy(c)
        H.hear_model_destroy(self.model)
        H.hear_eval_keys_destroy(self.evk)
        H.hear_public_key_destroy(self.pk)
        H.hear_secret_key_destroy(self.sk)
        H.hear_context_destroy(self.ctx)


def test_two_ring_sizes_in_one_launch(H):
    small, large = Job(H, "small", 7), Job(H, "large", 12)      # 2 + 2 ciphertexts, ragged last ones
    mu = None
    try:
        mu = H.hear_multi_create([small.model, large.model], [small.evk, large.evk],
                                 [len(small.cts), len(large.cts)], [2.0 ** 40, 2.0 ** 40])
        ref = H.hear_evaluate(small.model, small.evk, small.cts) + H.hear_evaluate(large.model, large.evk, large.cts)
        for rep in range(2):
            outs = H.hear_multi_evaluate(mu, small.cts + large.cts)
            assert len(outs) == len(ref)
            for a, b in zip(outs, ref):
                assert H.hear_ciphertext_info(a) == H.hear_ciphertext_info(b)
                assert np.array_equal(H.hear_ciphertext_export(a), H.hear_ciphertext_export(b))
            ns = len(small.cts)
            for job, part in ((small, outs[:ns]), (large, outs[ns:])):
                assert np.max(np.abs(job.logits(part) - job.w.fp64_forward(job.w.clips))) <= 2.0 ** -15
            for o in outs:
                H.hear_ciphertext_destroy(o)
        for o in ref:
            H.hear_ciphertext_destroy(o)
        low = H.hear_ciphertext_drop_level(small.cts[0], 3)
        with pytest.raises(H.HearError):
            H.hear_multi_evaluate(mu, [low] + small.cts[1:] + large.cts)
        H.hear_ciphertext_destroy(low)
        with pytest.raises(H.HearError):
            H.hear_multi_create([small.model], [large.evk], [1], [2.0 ** 40])   # keys of another context
    finally:
        if mu:
            H.hear_multi_destroy(mu)
        small.close()
        large.close()
