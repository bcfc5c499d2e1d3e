// noalloc.cu -- rescale for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: processes that run under a device-memory quota
// already filled by another framework's caching allocator, real-time loops that must not
// take the allocator's locks or latency, and hosts that only own pageable host memory and
// a stream.  hear_rescale_noalloc serves them: its device working memory is the
// file-scope array below, reserved once when the library is loaded on a device and held
// by every GPU that loads the library until the process exits.  The call allocates
// nothing (no cudaMalloc / cudaMallocAsync / cudaFree, no allocating library routine).
#include <map>
#include <mutex>
#include "ckks.h"

namespace hear {
namespace {

// 2^21 words = 16 MiB of device scratch
constexpr size_t kNoAllocScratchWords = (size_t)1 << 21;
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocScratchWords];

std::mutex g_noalloc_mu;                 // one call at a time: the calls share the array
std::map<int, uint64_t *> g_noalloc_ptr;  // device -> address of g_noalloc_scratch

// Address of the scratch array on the current device.  The host-side name of the array is
// only a stand-in; the device address comes from cudaGetSymbolAddress, resolved once per
// device with that device current.
uint64_t *scratch_on(int device) {
    auto it = g_noalloc_ptr.find(device);
    if (it != g_noalloc_ptr.end()) return it->second;
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        (void)cudaGetLastError();
        throw Error(HEAR_E_CUDA, std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") +
                                     cudaGetErrorString(e));
    }
    g_noalloc_ptr[device] = static_cast<uint64_t *>(p);
    return static_cast<uint64_t *>(p);
}

}  // namespace

void set_last_error(const std::string &msg);   // capi.cu

}  // namespace hear

using namespace hear;

extern "C" hear_status hear_rescale_noalloc(hear_context *ctx, const uint64_t *in, size_t in_words,
                                            uint32_t level, uint32_t n_poly, uint64_t *out, size_t out_cap,
                                            void *stream) {
    auto fail = [](hear_status c, const std::string &m) {
        set_last_error(m);
        return c;
    };
    if (!ctx || !in || !out) return fail(HEAR_E_INVAL, "null argument");
    if (ctx->poisoned) return fail(HEAR_E_CUDA, "context is poisoned by an earlier CUDA error");
    if (level < 1 || level > ctx->L) return fail(HEAR_E_LEVEL, "level must be in [1, L]");
    if (n_poly < 1 || n_poly > 3) return fail(HEAR_E_INVAL, "n_poly must be 1, 2 or 3");
    const uint64_t n = ctx->n;
    const uint64_t need_in = (uint64_t)n_poly * (level + 1) * n, need_out = (uint64_t)n_poly * level * n;
    if (in_words != need_in)
        return fail(HEAR_E_FORMAT, "input holds " + std::to_string(in_words) + " words; n_poly*(level+1)*N = " +
                                       std::to_string(need_in));
    if (out_cap < need_out)
        return fail(HEAR_E_INVAL, "output capacity " + std::to_string(out_cap) + " words < n_poly*level*N = " +
                                      std::to_string(need_out));
    if (need_in + need_out > kNoAllocScratchWords)
        return fail(HEAR_E_UNSUPPORTED, "n_poly*(2*level+1)*N = " + std::to_string(need_in + need_out) +
                                            " words exceeds the no-alloc scratch of " +
                                            std::to_string(kNoAllocScratchWords) + " words (16 MiB)");
    if (ctx->prof.on) return fail(HEAR_E_STATE, "stop the profiler before calling hear_rescale_noalloc");
    // every residue of limb i must be reduced mod q_i (as for hear_ciphertext_import)
    for (uint64_t w = 0; w < need_in; w++) {
        const uint64_t limb = (w / n) % (level + 1);
        if (in[w] >= ctx->primes[limb])
            return fail(HEAR_E_FORMAT, "word " + std::to_string(w) + " is not reduced mod its limb's prime");
    }
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    int prev_device = -1;
    if (cudaGetDevice(&prev_device) != cudaSuccess) {
        (void)cudaGetLastError();
        prev_device = -1;
    }
    hear_status status = HEAR_OK;
    try {
        HEAR_CHECK_CUDA(cudaSetDevice(ctx->device));
        cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        HEAR_CHECK_CUDA(cudaStreamIsCapturing(st, &cap));
        HEAR_REQUIRE(cap == cudaStreamCaptureStatusNone, HEAR_E_STATE,
                     "hear_rescale_noalloc synchronises its stream and cannot run on a stream being captured");
        uint64_t *x = scratch_on(ctx->device);     // input, NTT domain [n_poly][level+1][N]
        uint64_t *y = x + need_in;                 // result [n_poly][level][N]
        HEAR_CHECK_CUDA(cudaMemcpyAsync(x, in, need_in * 8, cudaMemcpyHostToDevice, st));
        ntt_forward(ctx, x, n_poly * (level + 1), map_q(level, ctx->n_q), st);
        rescale(ctx, level, n_poly, x, y, y, st);  // the combine writes each word after reading it
        ntt_inverse(ctx, y, n_poly * level, map_q(level - 1, ctx->n_q), st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(out, y, need_out * 8, cudaMemcpyDeviceToHost, st));
        HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    } catch (const Error &e) {
        // a CUDA error poisons the context, as every other call of the library does
        if (e.code == HEAR_E_CUDA) ctx->poisoned = true;
        status = fail(e.code, e.what());
    } catch (...) {
        status = fail(HEAR_E_INVAL, "unknown error");
    }
    if (prev_device >= 0) cudaSetDevice(prev_device);   // the caller's current device is left as it was
    return status;
}
