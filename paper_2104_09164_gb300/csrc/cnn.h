// cnn.h -- the encrypted skeleton CNN (internal): a plan of slot-level operations built from
// the layer list of hear_cnn_create and evaluated on a batch of samples.
#pragma once
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>
#include "ckks.h"

struct hear_cnn {
    enum OpKind : uint32_t { kDiag = HEAR_CNN_OP_DIAG, kPack = HEAR_CNN_OP_PACK, kRotsum = HEAR_CNN_OP_ROTSUM,
                             kQuad = HEAR_CNN_OP_QUAD, kBias = HEAR_CNN_OP_BIAS };
    struct Op {
        uint32_t kind = 0;
        uint32_t n_in = 0, n_out = 0;              // ciphertexts per sample before / after
        uint32_t level_in = 0, level_out = 0;
        // kDiag: out_j = rescale(sum_g rho^g(sum_(b,i) pt[g][j][b][i] (.) rho^b(x_i)))
        std::vector<int32_t> babies, giants;       // sorted slot amounts in [0, N/2); [0] = 0
        hear::DevBuf pts;                          // [giants][n_out][babies][n_in][L1][N] Montgomery
        // kPack: out_t = sum_p rho^(-offs[p])(rescale(x_(t n_p + p) (.) mask))
        hear::DevBuf mask;                         // [L1][N] Montgomery
        std::vector<int32_t> offs;
        // kRotsum: x <- x + rho^s(x)
        std::vector<int32_t> steps;
        // kQuad: A Montgomery [n_in][L1][N]; B, C slot vectors per ciphertext (encoded at
        // the scales the evaluation reaches); kBias: slot vector (one)
        hear::DevBuf A;
        std::vector<double> B, C, bias;            // [n_in][N/2] / [N/2]
    };
    // CUDA graph of operations [op0, op1) on C samples with given keys and input scale,
    // replayed from a fixed input / output workspace
    struct Plan {
        uint64_t evk_serial = 0;
        size_t op0 = 0, op1 = 0;
        uint32_t C = 0;
        double scale_in = 0, scale_out = 0;
        hear::DevBuf X, Y;
        cudaGraphExec_t exec = nullptr;
        cudaEvent_t done = nullptr;
        uint64_t launches = 0;
        ~Plan();
    };
    mutable std::mutex plan_mu;
    mutable std::vector<std::unique_ptr<Plan>> plans;
    hear_context *ctx = nullptr;
    std::vector<Op> ops;
    std::vector<uint32_t> op_layer;                // layer each operation comes from
    std::vector<uint32_t> out_slots;
    std::vector<int32_t> rotations;
    uint32_t in_kind = 0, in_c = 0, in_dist = 0, in_h = 0, in_w = 0, in_pitch = 0;
    // plaintexts whose scale depends on the input scale: (op index, scale at the op) ->
    // [B | C | bias] plaintexts (normal NTT form)
    mutable std::mutex mu;
    mutable std::map<std::pair<size_t, double>, hear::DevBuf> scaled;
};

namespace hear {

hear_cnn *cnn_create(hear_context *c, const hear_cnn_input *in, const hear_cnn_layer *layers, size_t n_layers);
// scale after ops [op0, op1) for a given scale at op0
double cnn_scale_after(const hear_cnn *m, size_t op0, size_t op1, double scale);
// run ops [op0, op1) on x [n_in(op0)][C][2][L1][N]; returns [n_out(op1-1)][C][2][L1'][N]
DevBuf cnn_evaluate(const hear_cnn *m, const hear_eval_keys *evk, size_t op0, size_t op1, const uint64_t *x,
                    uint32_t C, double scale_in, double *scale_out, cudaStream_t st);
// graph plan for (evk, op0, op1, C, scale_in): one direct warm-up run (builds every table the
// capture needs), then stream capture; the caller fills plan->X, launches plan->exec and
// reads plan->Y.  Caller holds m->plan_mu.
hear_cnn::Plan *cnn_graph_plan(const hear_cnn *m, const hear_eval_keys *evk, size_t op0, size_t op1, uint32_t C,
                               double scale_in, cudaStream_t st);
// slot vector of the input ciphertext(s) of one sample: [n_in][N/2]
std::vector<double> cnn_pack_input(const hear_cnn *m, const double *x);

}  // namespace hear
