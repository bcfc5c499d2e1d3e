// ckks.h -- batched RNS-CKKS operations and the encoded network (internal).
#pragma once
#include <map>
#include <memory>
#include <mutex>
#include <vector>
#include "internal.h"
#include "kernels.cuh"
#include "encode.h"

// Encoded network (Methods, "Non-convolutional layers" and "Algorithmic and cryptographic
// optimizations").
struct hear_model {
    struct Fc {
        uint32_t d_out = 0, d_in = 0, D = 0, n1 = 0, n2 = 0, level = 0;
        bool dh = false;                            // hoisted ModDown: babies and inner sums over Q_l u P
        hear::DevBuf pts;                           // [n2*n1][level+1 (+K if dh)][N] Montgomery, zero = no diagonal
        hear::DevBuf pmod;                          // dh: ([P]_{q_t}, Shoup) for t <= level
        std::vector<double> bias;                   // d_out bias values (empty: none), added after the
                                                    // rotate-and-sum at the output level and scale
        std::vector<std::vector<int32_t>> rotsum;   // rotate-and-sum rounds (slot steps, hoisted per round)
    };
    struct Layer {
        uint32_t kind = 0;
        uint32_t level_in = 0, level_out = 0;
        Fc fc, fc2;                                 // FC; FC_SQ_FC: fc = W1, fc2 = collapsed U
        std::vector<std::vector<int32_t>> final_rotsum;   // FC_SQ_FC: sum over r (rounds)
    };
    // CUDA graph of one evaluation (layers [l0, l1) for n_ct ciphertexts with given keys and
    // input scale), replayed from a fixed input/output workspace
    struct Plan {
        uint64_t evk_serial = 0;   // keys the graph reads (never reused after they are freed)
        size_t l0 = 0, l1 = 0;
        uint32_t n_ct = 0, level_out = 0;
        uint32_t slot = 0;         // independent copies for concurrent users (server slots)
        bool host_io = false;      // X / Y in the coefficient domain (graph_plan)
        double scale_in = 0, scale_out = 0;
        hear::DevBuf X, Y;
        cudaGraphExec_t exec = nullptr;
        cudaEvent_t done = nullptr;
        uint64_t launches = 0;
        ~Plan();
    };
    hear_context *ctx = nullptr;
    uint32_t clip_dim = 0, k = 0, M = 0;
    uint32_t rotsum_radix = 8;                      // copies folded per rotate-and-sum round
    uint32_t fc_n1 = 0;                             // FC baby steps (0 = smallest power of two with n1^2 >= D)
    bool hoist_moddown = false;                     // FC babies kept over Q_l u P, one ModDown per giant sum
    bool hoist_sums = false;                        // giant sums and rotate-and-sum rounds ModDowned once
    hear::DevBuf pmod_all;                          // ([P]_{q_t}, Shoup) for t < n_q
    // bias plaintexts (normal NTT form at the FC's output level) per (layer, output scale):
    // built before the first launch of an evaluation at that scale, never inside a capture
    mutable std::mutex bias_mu;
    mutable std::map<std::pair<size_t, uint64_t>, hear::DevBuf> bias_pts;
    mutable std::mutex plan_mu;
    mutable std::vector<std::unique_ptr<Plan>> plans;
    std::vector<Layer> layers;
    std::vector<uint32_t> out_pos;
    std::vector<int32_t> rotations;
};

// Several networks (own contexts, possibly different ring sizes, one device) evaluated by one
// CUDA graph whose branches -- one per job, captured on forked streams -- run concurrently.
struct hear_multi {
    std::vector<const hear_model *> models;
    std::vector<const hear_eval_keys *> evks;
    std::vector<uint32_t> n_ct, level_in, level_out;
    std::vector<double> scale_in, scale_out;
    std::vector<hear::DevBuf> X, Y;    // per job: input / output batches the graph reads / writes
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;        // the last launch finished with X / Y
    uint64_t launches = 0;
    ~hear_multi();
};

namespace hear {

void forget_encoder(hear_context *ctx);
std::shared_ptr<EncoderTables> encoder(hear_context *ctx);
std::vector<uint64_t> make_cdt(double sigma);
void build_context(hear_context *c, const hear_params_desc *d, int device);

uint32_t galois_of(const hear_context *c, int64_t step);
uint32_t galois_inverse(const hear_context *c, uint32_t g);

// keygen / encryption / decryption
void keygen(hear_context *c, uint64_t seed, const int32_t *steps, size_t n_steps, hear_secret_key **sk,
            hear_public_key **pk, hear_eval_keys **evk);
hear_ciphertext *encrypt_slots(hear_context *c, const hear_public_key *pk, const double *z, double scale,
                               uint64_t seed, uint64_t ct_id, cudaStream_t st);
// the same from an encoded message m (N integer coefficients)
hear_ciphertext *encrypt_encoded(hear_context *c, const hear_public_key *pk, const int64_t *m, double scale,
                                 uint64_t seed, uint64_t ct_id, cudaStream_t st);
void decrypt_slots(hear_context *c, const hear_secret_key *sk, const hear_ciphertext *ct, double *out);

// batched primitives on contiguous batches [n_ct][n_poly][level+1][N]
struct Rot {
    const uint64_t *key;
    uint32_t galois;
};
// out[r*n_ct + c] = rho_r(x[c]) for every rotation r, sharing one ModUp of the c1 of each
// x[c] (hoisting); out is contiguous [R][n_ct][2][level+1][N]
void rotate_hoisted(hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *x,
                    const std::vector<Rot> &rots, uint64_t *out, cudaStream_t st);
// the hoisted rotations before ModDown: out_ext [R][n_ct][2][W][N] over Q_l u P holds
// (P sigma_r(c0) + u0, u1); pmod = ([P]_{q_t}, Shoup) pairs
void rotate_hoisted_ext(hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *x, const std::vector<Rot> &rots,
                        uint64_t *out_ext, const uint64_t *pmod, cudaStream_t st);
// out[r*C + c] = rho_r(x[r*C + c]): job r rotates its C ciphertexts with rots[r]
void rotate_each(hear_context *c, uint32_t level, uint32_t R, uint32_t C, const uint64_t *x,
                 const std::vector<Rot> &rots, uint64_t *out, cudaStream_t st);
// the same before ModDown: out_ext [R][C][2][W][N] over Q_l u P holds (P sigma_r(c0) + u0, u1)
void rotate_each_ext(hear_context *c, uint32_t level, uint32_t R, uint32_t C, const uint64_t *x,
                     const std::vector<Rot> &rots, uint64_t *out_ext, const uint64_t *pmod, cudaStream_t st);
// tensor + relinearise (no rescale): out [n_ct][2][level+1][N]
void mul_relin(hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *a, const uint64_t *b,
               const uint64_t *relin_key, uint64_t *out, cudaStream_t st);
// relinearise degree-2 ciphertexts d3 [n_ct][3][level+1][N] -> out [n_ct][2][level+1][N]
void relin3(hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *d3, const uint64_t *relin_key,
            uint64_t *out, cudaStream_t st);

// encoded plaintext helpers
DevBuf encode_plain(hear_context *c, const double *z, double scale, uint32_t level, cudaStream_t st,
                    bool mont = true);

// network
// copies folded per rotate-and-sum round by default (measured on the small network at batch
// 1: 1.45 / 1.20 / 1.19 / 1.22 ms for radix 2 / 4 / 8 / 16)
constexpr uint32_t kDefaultRotsumRadix = 8;
// the network evaluated from input ciphertexts at start_level (every plaintext encoded at
// the level where it is used)
hear_model *model_create(hear_context *c, const hear_layer_desc *layers, size_t n_layers, uint32_t clip_dim,
                         uint32_t start_level, uint32_t rotsum_radix = kDefaultRotsumRadix, uint32_t fc_n1 = 0,
                         bool hoist_moddown = false, bool hoist_sums = false);
// evaluate layers [l0, l1) on a batch x at the first layer's level; returns the output batch
DevBuf evaluate_batch(const hear_model *m, const hear_eval_keys *evk, size_t l0, size_t l1, const uint64_t *x,
                      uint32_t n_ct, uint32_t *level_out, double scale_in, double *scale_out, cudaStream_t st);
// graph plan for (evk, l0, l1, n_ct, scale_in): built on first use (one direct warm-up run,
// then stream capture); the caller fills plan->X, launches plan->exec and reads plan->Y.
// host_io: X and Y hold coefficient-domain ciphertexts (the forward NTT of X and the inverse
// NTT into Y are part of the graph, X is transformed in place), for callers that copy from
// and to host memory
hear_model::Plan *graph_plan(const hear_model *m, const hear_eval_keys *evk, size_t l0, size_t l1, uint32_t n_ct,
                             double scale_in, cudaStream_t st, uint32_t slot = 0, bool host_io = false);
// the one-launch graph of several whole-network jobs (see hear_multi); one direct warm-up run
// of every job on `st` first (builds the tables the capture needs)
hear_multi *multi_create(const hear_model *const *models, const hear_eval_keys *const *evks, size_t n_jobs,
                         const uint32_t *n_ct, const double *scales, cudaStream_t st);

}  // namespace hear
