// simd.h -- slot-batched evaluation of the FC / x^2 networks (internal): one clip per slot,
// one ciphertext per feature, FC layers as plaintext scalars times ciphertexts.
#pragma once
#include <vector>
#include "ckks.h"

struct hear_simd_model {
    struct Layer {
        uint32_t kind = 0;                 // HEAR_LAYER_FC / _SQUARE / _FC_SQ_FC
        uint32_t n_in = 0, n_out = 0;      // ciphertexts before / after
        uint32_t level_in = 0, level_out = 0;
        // FC and FC_SQ_FC: the matrix product of M x K scalars (rows padded to Mpad) with the
        // K input ciphertexts; FC_SQ_FC rows are (r, c) -> W1[r] for r*d2 + c, then
        // W2[c, r] W1[r] for d1*d2 + r*d2 + c
        uint32_t M = 0, Mpad = 0, K = 0, d1 = 0, d2 = 0;
        hear::DevBuf a;                    // u32 pieces, limb t at a_off[t]: [3 planes][K][Mpad]
        hear::DevBuf a_off;                // u64 [L1] offsets into a
        hear::DevBuf consts;               // per-limb reduction constants
        std::vector<uint8_t> limbs_narrow, limbs_wide;   // primes below 2^42 / below 2^62
    };
    hear_context *ctx = nullptr;
    uint32_t d_in = 0, d_out = 0, level_in = 0, level_out = 0;
    std::vector<Layer> layers;
};

// a batch of ciphertexts stored contiguously in HBM: [n_ct][2][level+1][N], NTT domain
struct hear_simd_batch {
    hear_context *ctx = nullptr;
    uint32_t n_ct = 0, level = 0;
    double scale = 1.0;
    hear::DevBuf d;
};

namespace hear {

// lane operations per second of the integer multiply-add (kind 0: mad.wide.u32, 1: mad.lo.u32)
// measured by a throughput kernel over every SM
double imad_peak(hear_context *c, int kind, uint32_t iters);

// exact round(w * q) with ties away from zero (|w q| < 2^62)
int64_t round_scalar(double w, uint64_t q);

// dynamic shared memory of the matrix-product kernels on the current device; called once
// per context at creation
void simd_setup();
hear_simd_model *simd_model_create(hear_context *c, const hear_layer_desc *layers, size_t n_layers,
                                   uint32_t level);
// evaluate the network on x [d_in][2][level_in+1][N]; returns [d_out][2][level_out+1][N]
DevBuf simd_evaluate(const hear_simd_model *m, const hear_eval_keys *evk, const uint64_t *x, double scale_in,
                     double *scale_out, cudaStream_t st);

}  // namespace hear
