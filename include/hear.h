/*
 * hear.h -- C ABI of the GB300 (sm_103a) RNS-CKKS library for encrypted inference in the
 * style of HEAR / Fast-HEAR ("Secure Human Action Recognition by Encrypted Neural
 * Network Inference", arXiv 2104.09164).
 *
 * The calls follow the paper's statement of the problem (Results, "Overview of HEAR",
 * and the Fig. 1 caption): the monitoring provider generates the keys (secret key,
 * public key, evaluation keys for ciphertext products and rotations) and decrypts
 * results; the end-user encrypts with the public key; the cloud evaluates the network on
 * ciphertexts with the evaluation keys only.  The scheme is the RNS variant of CKKS
 * (Methods, "Algorithmic and cryptographic optimizations").
 *
 * Conventions
 *   - Every call returns hear_status: HEAR_OK (0) or a negative error code; the
 *     thread-local message of the last error is available from hear_last_error().
 *   - Handles are created by the library and released by the caller with the matching
 *     *_destroy call (NULL is accepted and ignored).
 *   - Host arrays passed in are borrowed for the duration of the call only.  Output arrays
 *     are caller-allocated with a capacity `cap` (in elements) and the count written to
 *     *n; a short capacity returns HEAR_E_INVAL with the required count in *n.
 *   - `stream` is a cudaStream_t (NULL = the context's own stream).  Calls that return
 *     device-resident handles enqueue their work on that stream; calls that fill host
 *     arrays synchronise it before returning.  A ciphertext's memory comes from the
 *     stream-ordered allocator of the stream it was produced on and goes back to it when
 *     the handle is destroyed, so that stream must outlive the handle, and work queued on
 *     other streams must be complete (or ordered before that stream) when it is destroyed.
 *   - Ciphertexts live in device memory (HBM) in the library's NTT domain, laid out as
 *     uint64_t[n_poly][level+1][N], one word per residue.  Exported/imported ciphertexts
 *     use the coefficient domain with the same layout.
 *   - Keys and models are immutable after creation and may be shared by concurrent
 *     evaluations on different streams.  After a CUDA error the context is poisoned:
 *     every later call on it returns HEAR_E_CUDA.
 *   - No C++ exception crosses this interface and nothing aborts the process.
 *   - There is no CPU fallback: all ring arithmetic runs in the library's CUDA kernels.
 */
#ifndef HEAR_H
#define HEAR_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int hear_status;
#define HEAR_OK 0
#define HEAR_E_INVAL (-1)       /* bad argument (pointer, size, capacity)            */
#define HEAR_E_NOMEM (-2)       /* host or device allocation failed                   */
#define HEAR_E_CUDA (-3)        /* CUDA error; the context is poisoned                */
#define HEAR_E_LEVEL (-4)       /* ciphertext has no level left for the operation     */
#define HEAR_E_SCALE (-5)       /* operands at different scales or levels             */
#define HEAR_E_NOKEY (-6)       /* missing rotation or relinearisation key            */
#define HEAR_E_STATE (-7)       /* handle from another context / wrong kind           */
#define HEAR_E_FORMAT (-8)      /* malformed import buffer                            */
#define HEAR_E_UNSUPPORTED (-9) /* parameter outside the supported range              */
#define HEAR_E_TIMEOUT (-10)    /* a bounded wait ran out before the work finished    */
#define HEAR_E_BUSY (-11)       /* admission refused: queue or staging buffers full   */

typedef struct hear_context hear_context;
typedef struct hear_secret_key hear_secret_key;
typedef struct hear_public_key hear_public_key;
typedef struct hear_eval_keys hear_eval_keys;
typedef struct hear_ciphertext hear_ciphertext;
typedef struct hear_model hear_model;
typedef struct hear_cnn hear_cnn;
typedef struct hear_multi hear_multi;
typedef struct hear_simd_model hear_simd_model;
typedef struct hear_simd_batch hear_simd_batch;

/* Encryption parameters.  The ciphertext modulus is Q = q_0 * ... * q_{n_q-1} (top level
 * L = n_q - 1); the n_p special primes p_0..p_{K-1} are used by key switching only.
 * Prime rule: for each bit size in the order q_0, q_1.., p_0.. take the largest prime
 * below 2^bits that is 1 mod 2N and not yet taken.  Hybrid key switching uses digits of
 * alpha consecutive limbs from q_0; alpha must equal n_p (0 selects that value; any other
 * value returns HEAR_E_UNSUPPORTED, because a digit modulus above P multiplies the
 * key-switching error by Q_j / P).  Supported: log_n in [11, 16], bit sizes in
 * [log_n + 2, 60], n_q + n_p <= 48.  sigma: standard deviation of the discrete Gaussian
 * errors (tail cut at floor(6 sigma)). */
typedef struct hear_params_desc {
    uint32_t log_n;
    uint32_t n_q;
    const uint32_t *q_bits;
    uint32_t n_p;
    const uint32_t *p_bits;
    double log2_scale;  /* encoding scale of fresh inputs, e.g. 40 */
    double sigma;       /* e.g. 3.2 */
    uint32_t alpha;     /* limbs per key-switching digit: n_p, or 0 for n_p */
} hear_params_desc;

const char *hear_last_error(void);

/* ---- context: primes, NTT tables and basis-conversion constants on `device` ---- */
hear_status hear_context_create(const hear_params_desc *params, int cuda_device, hear_context **out);
void hear_context_destroy(hear_context *ctx);
/* primes in chain order q_0..q_{n_q-1}, p_0..p_{K-1} */
/* Route the context's device allocations through the caller's allocator: while an ABI call
 * of this context runs, every device allocation it makes on the calling thread calls
 * alloc(bytes, stream, user) (stream = the CUDA stream the memory is for, null = synchronous
 * use) and is released later by free(ptr, stream, user).  Memory a CUDA graph owns (allocated
 * inside a stream capture) and the server worker thread's memory stay with the stream-ordered
 * pool.  alloc returns null on failure: the call fails with HEAR_E_NOMEM and the context stays
 * usable.  free is stream-ordered: work already queued on `stream` may still use the block
 * when free(ptr, stream, user) is called, so the block may be handed out again only to work
 * ordered after that stream's pending work (as PyTorch's caching allocator does); for a null
 * stream the block must not be reused before the device is synchronised.  Both functions
 * null = back to the pool; every pair installed must stay valid until the context and
 * everything made with it are destroyed (memory allocated through a pair is released
 * through it). */
hear_status hear_set_allocator(hear_context *ctx, void *(*alloc)(size_t bytes, void *stream, void *user),
                               void (*free)(void *ptr, void *stream, void *user), void *user);
hear_status hear_context_primes(const hear_context *ctx, uint64_t *out, size_t cap, size_t *n);
/* discrete-Gaussian CDT thresholds used by the samplers (for cross-checking) */
hear_status hear_context_cdt(const hear_context *ctx, uint64_t *out, size_t cap, size_t *n);

/* ---- key generation (monitoring provider).  All randomness is drawn from the
 * counter-based ChaCha20 generator (RFC 8439) keyed by `seed`.  One rotation key is
 * generated per entry of rot_steps (left rotation by that many slots); duplicates are
 * ignored.  The keys stay resident in device memory. ---- */
hear_status hear_keygen(hear_context *ctx, uint64_t seed, const int32_t *rot_steps, size_t n_steps,
                        hear_secret_key **sk, hear_public_key **pk, hear_eval_keys **evk);
void hear_secret_key_destroy(hear_secret_key *);
void hear_public_key_destroy(hear_public_key *);
void hear_eval_keys_destroy(hear_eval_keys *);
/* the ternary secret s (N coefficients in {-1,0,1}) -- test and audit use only */
hear_status hear_secret_key_export(const hear_secret_key *sk, int8_t *out, size_t cap, size_t *n);
/* public key (b, a) over Q_L, coefficient domain uint64[2][n_q][N] */
hear_status hear_public_key_export(const hear_public_key *pk, uint64_t *out, size_t cap, size_t *n);
/* switching key for `galois` (1 = relinearisation key, else the key of X -> X^galois),
 * coefficient domain uint64[dnum][2][n_q+n_p][N] */
hear_status hear_eval_key_export(const hear_eval_keys *evk, uint32_t galois, uint64_t *out, size_t cap,
                                 size_t *n);

/* ---- encoding / encryption (end-user) ---- */
/* round(scale * tau^-1(z)) for n_slots = N/2 real values (canonical embedding, slot j at
 * the root exp(i*pi*5^j/N)), computed in double-double arithmetic, ties away from zero */
hear_status hear_encode(const hear_context *ctx, const double *z, size_t n_slots, double scale,
                        int64_t *m_out, size_t cap, size_t *n);
/* encrypt N/2 slot values at `scale` (0 = the context's default scale) at the top level.
 * The encryption randomness is stream `ct_id` of `seed`. */
hear_status hear_encrypt(hear_context *ctx, const hear_public_key *pk, const double *z, size_t n_slots,
                         double scale, uint64_t seed, uint64_t ct_id, hear_ciphertext **out, void *stream);
/* Data encryption with interlaced copies (Methods, "Data encryption"): n_clips row-major
 * clips of clip_dim values (clip_dim a power of two dividing N/2); with k = (N/2)/clip_dim
 * lanes, slot p*k + c holds clip (c mod n_clips)[p]; requires 1 <= n_clips <= k. */
hear_status hear_encrypt_clips(hear_context *ctx, const hear_public_key *pk, const double *clips,
                               size_t n_clips, size_t clip_dim, uint64_t seed, uint64_t ct_id,
                               hear_ciphertext **out, void *stream);
/* decrypt + decode to N/2 real slot values */
hear_status hear_decrypt(hear_context *ctx, const hear_secret_key *sk, const hear_ciphertext *ct,
                         double *out, size_t cap, size_t *n);
void hear_ciphertext_destroy(hear_ciphertext *);
hear_status hear_ciphertext_info(const hear_ciphertext *ct, uint32_t *level, uint32_t *n_poly, double *scale);
/* coefficient domain uint64[n_poly][level+1][N] */
hear_status hear_ciphertext_export(const hear_ciphertext *ct, uint64_t *out, size_t cap, size_t *n);
hear_status hear_ciphertext_import(hear_context *ctx, const uint64_t *words, size_t n_words, uint32_t level,
                                   uint32_t n_poly, double scale, hear_ciphertext **out, void *stream);

/* ---- primitive homomorphic operations (cloud) ---- */
/* rho^step: left rotation of the slots by `step` (negative = right), via X -> X^(5^step) */
hear_status hear_rotate(const hear_eval_keys *evk, const hear_ciphertext *ct, int32_t step,
                        hear_ciphertext **out, void *stream);
/* several rotations of one ciphertext sharing a single ModUp (hoisting, Methods,
 * "Algorithmic and cryptographic optimizations" item (i)); out[i] = rho^steps[i](ct) */
hear_status hear_rotate_hoisted(const hear_eval_keys *evk, const hear_ciphertext *ct, const int32_t *steps,
                                size_t n_steps, hear_ciphertext **out, void *stream);
/* divide by the last prime and drop it (lazy rescaling uses it once per sum) */
hear_status hear_rescale(const hear_ciphertext *ct, hear_ciphertext **out, void *stream);
/* the same ciphertext over Q_level (level <= its level): the residues of the primes above
 * `level` are discarded, no division, the scale is unchanged.  Evaluating a network from
 * the lowest level its depth needs (minimal start level) makes every later operation work
 * on fewer limbs; the plaintexts of a model built for that level carry only those limbs
 * (Methods, "Algorithmic and cryptographic optimizations", level-aware encoding). */
hear_status hear_ciphertext_drop_level(const hear_ciphertext *ct, uint32_t level, hear_ciphertext **out,
                                       void *stream);
hear_status hear_add(const hear_ciphertext *a, const hear_ciphertext *b, hear_ciphertext **out, void *stream);
/* MultPlain(ct, pt): multiply by the plaintext encoding of N/2 slot values at pt_scale
 * (level-aware: the plaintext carries only the limbs of ct's level) -- no rescale */
hear_status hear_mulplain(const hear_ciphertext *ct, const double *z, size_t n_slots, double pt_scale,
                          hear_ciphertext **out, void *stream);
/* ciphertext product: tensor, then relinearisation with the s^2 key -- no rescale */
hear_status hear_multiply_relin(const hear_eval_keys *evk, const hear_ciphertext *a, const hear_ciphertext *b,
                                hear_ciphertext **out, void *stream);

/* ---- network (cloud) ---- */
#define HEAR_LAYER_FC 1          /* y = W x (d_out x d_in, row-major), optional bias       */
#define HEAR_LAYER_SQUARE 2      /* y = x^2 (polynomial activation)                       */
#define HEAR_LAYER_FC_SQ_FC 3    /* y = W2 (W1 x)^2 evaluated as one collapsed quadratic    */
typedef struct hear_layer_desc {
    uint32_t kind;
    uint32_t d_out, d_in;   /* W: d_out x d_in; powers of two with d_out | d_in            */
    const double *w;        /* row-major                                                   */
    const double *bias;     /* d_out values or NULL (FC only): added after the rotate-and-
                             * sum as a plaintext b[p mod d_out] in every slot p*k + c,
                             * encoded at the output's level and scale                    */
    uint32_t d_out2;        /* FC_SQ_FC: W2 is d_out2 x d_out                               */
    const double *w2;
} hear_layer_desc;

/* Encode the network for ciphertexts packed by hear_encrypt_clips with clip_dim inputs.
 * FC layers are evaluated as baby-step/giant-step diagonal products: D = d_out extended
 * diagonals diag_i[p] = W[p mod d_out][(p+i) mod d_in], n1 = smallest power of two with
 * n1^2 >= D, n2 = ceil(D/n1); hoisted baby rotations rho^(i k), plaintexts pre-rotated by
 * rho^(-j n1 k) and encoded at the level of use with scale q_level, non-hoisted giant
 * rotations rho^(j n1 k), one rescale, then the sum of the d_in/d_out copies rho^(j d_out k)
 * in rounds of up to 8 (rotsum_radix) copies whose rotations share one ModUp
 * (Methods, "Algorithmic and cryptographic optimizations"; "Non-convolutional layers"). */
hear_status hear_model_create(hear_context *ctx, const hear_layer_desc *layers, size_t n_layers,
                              uint32_t clip_dim, hear_model **out);
/* the same network for input ciphertexts at `level` (1 <= level <= L; the network's depth
 * must fit): every plaintext is encoded with the limbs of the level where it is used */
hear_status hear_model_create_at_level(hear_context *ctx, const hear_layer_desc *layers, size_t n_layers,
                                       uint32_t clip_dim, uint32_t level, hear_model **out);
/* model options: level = input level (0 = the top level); rotsum_radix = copies folded
 * per rotate-and-sum round (0 = the default 8; 2 is the plain log2-depth tree; r > 2 folds
 * r copies with r - 1 rotations that share one ModUp (hoisting), cutting the sequential
 * rounds to ceil(log_r) at the cost of more rotation keys; a power of two <= 64).
 * hear_model_create and hear_model_create_at_level use the default. */
typedef struct hear_model_opts {
    uint32_t level;
    uint32_t rotsum_radix;
    uint32_t fc_n1;          /* FC baby steps (power of two; 0 = smallest n1 with n1^2 >= d_out) */
    uint32_t hoist_moddown;  /* 1: FC baby rotations kept over Q_l u P (baby 0 = P x), inner sums
                              * with plaintexts over Q_l u P, one ModDown per giant-step sum --
                              * n2 instead of n1 ModDowns per ciphertext (FC layers only) */
    uint32_t hoist_sums;     /* 1: rotations whose results are summed stay over Q_l u P and the
                              * sum is ModDowned once -- the giant-step rotations of an FC layer
                              * together with inner sum 0 (one ModDown instead of n2 - 1), and
                              * each rotate-and-sum round (one instead of radix - 1); the same
                              * rotation keys, results differ from the unhoisted form only by
                              * ModDown rounding */
} hear_model_opts;
hear_status hear_model_create_ex(hear_context *ctx, const hear_layer_desc *layers, size_t n_layers,
                                 uint32_t clip_dim, const hear_model_opts *opts, hear_model **out);
/* input and output level of a model */
hear_status hear_model_levels(const hear_model *m, uint32_t *level_in, uint32_t *level_out);
void hear_model_destroy(hear_model *);
/* rotation steps (slots) the model needs keys for */
hear_status hear_model_rotations(const hear_model *m, int32_t *steps, size_t cap, size_t *n);
/* pos of logit c in the pos space (slot = pos * k + clip) */
hear_status hear_model_output_positions(const hear_model *m, uint32_t *pos, size_t cap, size_t *n);
/* evaluate the whole network on n_ct ciphertexts (one batch; all at the top level) */
hear_status hear_evaluate(const hear_model *m, const hear_eval_keys *evk, hear_ciphertext *const *in, size_t n_ct,
                          hear_ciphertext **out, void *stream);
/* several networks -- own contexts, possibly different ring sizes (e.g. the small N = 2^14
 * and the large N = 2^15 network), one device -- evaluated by ONE CUDA-graph launch whose
 * branches run concurrently: job i evaluates models[i] with evks[i] on n_ct[i] ciphertexts at
 * the model's input level and scales[i].  Creating it runs every job once and captures the
 * graph; destroy it before any of its models or keys. */
hear_status hear_multi_create(const hear_model *const *models, const hear_eval_keys *const *evks, size_t n_jobs,
                              const uint32_t *n_ct, const double *scales, hear_multi **out);
/* in: the jobs' input ciphertexts concatenated (job 0's n_ct[0] first); out (caller array of
 * the same length): the result ciphertexts in the same order, as hear_evaluate gives them;
 * stream null = the first job's context stream */
hear_status hear_multi_evaluate(hear_multi *mu, hear_ciphertext *const *in, hear_ciphertext **out, void *stream);
void hear_multi_destroy(hear_multi *mu);
/* evaluate layer `layer` only (input at that layer's level) */
hear_status hear_evaluate_layer(const hear_model *m, size_t layer, const hear_eval_keys *evk,
                                hear_ciphertext *const *in, size_t n_ct, hear_ciphertext **out, void *stream);
/* end-to-end from host buffers: n_ct input ciphertexts in the coefficient domain
 * (uint64[n_ct][2][l+1][N] at the model's input level l, `scale`) -> the result ciphertexts in the
 * coefficient domain (uint64[n_ct][2][level_out+1][N]); copies both ways are included */
hear_status hear_evaluate_host(const hear_model *m, const hear_eval_keys *evk, const uint64_t *in_words,
                               size_t n_ct, double scale, uint64_t *out_words, size_t cap, size_t *n,
                               uint32_t *level_out, double *scale_out, void *stream);

/* ---- continuous-batching server (cloud) ----
 * Requests carry ciphertexts in the coefficient domain in host memory (the format
 * hear_ciphertext_export produces; uint64[n_ct][2][L+1][N] at the top level, all at one
 * scale).  A worker thread admits pending requests in arrival order while the ciphertexts
 * in flight fit hbm_budget_bytes (each charged bytes_per_ciphertext: its share of the
 * evaluation's device work buffers plus input and output), packs up to max_batch
 * ciphertexts into one batch and runs it on one of n_slots streams, so batches admitted
 * while others run overlap on the device.  Each batch replays captured CUDA graphs of the
 * whole network (the first batch of each size captures them).  Results are the result
 * ciphertexts in the coefficient domain, uint64[n_ct][2][level_out+1][N]; they are
 * bit-identical to evaluating the request alone.  Host copies: a request's words are
 * copied once, at submit, into pinned staging buffers the server owns (staging_cts
 * ciphertexts), from which the batch is uploaded; results come back into pinned result
 * buffers and are copied once into the caller's array by poll / wait. */
typedef struct hear_server hear_server;
typedef struct hear_server_config {
    uint32_t max_batch;          /* ciphertexts per launch (>= 1)                         */
    uint32_t n_slots;            /* batches in flight, 1..8                               */
    uint64_t hbm_budget_bytes;   /* device bytes for the ciphertexts in flight            */
    uint32_t staging_cts;        /* pinned staging buffers, in ciphertexts, for queued and
                                    running requests (>= max_batch; 0 = the larger of
                                    4 n_slots max_batch and 64)                              */
    uint32_t max_pending;        /* queued requests beyond which submit is refused (0 = any) */
} hear_server_config;
typedef struct hear_server_counters {
    uint64_t requests_done, ciphertexts_done, clips_done, batches, pending;
    uint64_t max_in_flight_ciphertexts, bytes_per_ciphertext;
    double p50_ms, p99_ms, mean_ms;   /* submit -> result ready, completed requests      */
    uint64_t busy_refusals;           /* submits refused with HEAR_E_BUSY                 */
} hear_server_counters;
hear_status hear_server_create(const hear_model *m, const hear_eval_keys *evk, const hear_server_config *cfg,
                               hear_server **out);
/* queue a request of n_ct ciphertexts (n_clips clips, for the statistics); the words are
 * copied into the server's pinned staging buffers before the call returns.  HEAR_E_BUSY
 * (nothing queued) while the staging buffers cannot take n_ct more ciphertexts or
 * max_pending requests are queued: retry after results have been read. */
hear_status hear_server_submit(hear_server *s, const uint64_t *words, size_t n_ct, uint32_t n_clips, double scale,
                               uint64_t *request_id);
/* *done = 1 and the result copied to out (cap words, *n written) once the request is
 * complete (the id is then released); *done = 0 while it is queued or running */
hear_status hear_server_poll(hear_server *s, uint64_t request_id, uint64_t *out, size_t cap, size_t *n, int *done);
/* block until the request is complete (result copied to out as by poll, the id released)
 * or timeout_ms have passed: then HEAR_E_TIMEOUT, and the request stays queued or running
 * (wait or poll again later).  A failed request returns its error. */
hear_status hear_server_wait(hear_server *s, uint64_t request_id, uint32_t timeout_ms, uint64_t *out, size_t cap,
                             size_t *n);
/* paused != 0: admit no new batch (running batches finish; submits still queue) */
hear_status hear_server_pause(hear_server *s, int paused);
hear_status hear_server_stats(hear_server *s, hear_server_counters *stats);
/* waits for the batches in flight, drops queued requests; no other call on the server may
 * be in progress */
void hear_server_destroy(hear_server *s);

/* ---- skeleton CNN (cloud) ----
 * Methods, "Single-channel homomorphic convolutions", "Multi-channel homomorphic
 * convolutions" (Eq. conv), "Fast homomorphic convolutions", "Non-convolutional layers",
 * "Data encryption" and "Algorithmic and cryptographic optimizations" (full-step /
 * giant-step / baby-step strategies, hoisting, lazy rescaling, level-aware encoding).
 *
 * Slot layout.  dist = the smallest power of two >= h*w; the N/2 slots are cbar = N/2/dist
 * blocks of dist slots, each holding one channel map row-major with row pitch `pitch`
 * (map position (y, x) at block offset stride*(y*pitch + x); stride > 1 after pooling).
 * With c channels >= cbar, ciphertext i block m holds channel cbar*i + m (c must be a
 * multiple of cbar); with c < cbar (cbar a multiple of c) one ciphertext holds copies,
 * block m = channel m mod c.
 *
 * Layers.  A network may be given as trained (BN_QUAD, AVGPOOL, GAVGPOOL) and the library
 * collapses it (Methods, "Non-convolutional layers"): a block's convolution bias, batch
 * normalisation and quadratic activation become one per-channel quadratic, and the 1/2,
 * 1/4 or 1/(h*w) of average pooling move into the next linear layer's weights, computed in
 * IEEE double in the order A = (a*s)*s, B = ((2*a)*s)*t + b*s, C = ((a*t)*t + b*t) + c with
 * s = gamma / sqrt(var + eps), t = s*(bias - mean) + beta, conv weights w*f and FC weights
 * (w*f)/(h*w) (f = the pending pooling factor).  Or it may be given already collapsed
 * (QUAD, POOL, GAP):
 *   BN_QUAD  per channel of the preceding CONV: conv_bias (float64[c] or NULL = 0),
 *         bn_gamma, bn_beta, bn_mean, bn_var (float64[c]), bn_eps, then the activation
 *         act[0] z^2 + act[1] z + act[2]; becomes QUAD with (A, B, C) above.
 *   AVGPOOL  POOL whose 1/2 (1D) or 1/4 (2D) multiplies the next CONV's weights.
 *   GAVGPOOL GAP whose 1/(h*w) (map size at that point) divides the FC's weights.
 *   CONV  same-padded, stride-1 convolution, w = float64[c_out][c_in][f_h][f_w] (1D: f_h =
 *         1), c_out a multiple of cbar.  Rotation r + dist*l for tap (du, dv), r =
 *         stride*(du*pitch + dv), block shift l; the plaintexts carry the zero padding.
 *         fast = 1 (input punctured, stride > 1): merge-and-conquer -- pack n_P = (stride
 *         in 1D, stride^2 in 2D, at most the input ciphertext count, a power of two)
 *         punctured ciphertexts into one (mask plaintext, rescale, rotation by -phase,
 *         sum: one level), convolve, then rotate-and-sum over the phases (log2 n_P
 *         rotations).  Strategy: how each rotation a = b + g splits into a hoisted baby
 *         step b and a giant step g applied to the summed products:
 *           HEAR_STRATEGY_FULL   b = a, g = 0 (every rotated input precomputed)
 *           HEAR_STRATEGY_BABY   b = r, g = dist*l
 *           HEAR_STRATEGY_GIANT  b = dist*l, g = r
 *           HEAR_STRATEGY_HYBRID b = r + dist*(l mod n1), g = dist*n1*floor(l/n1)
 *   QUAD  per-channel a, b, c (float64[c]): x <- a x^2 + b x + c at the valid map
 *         positions, 0 elsewhere; two levels: u = rescale(x (.) a) + b, then
 *         rescale(relin(x * u)) + c.
 *   POOL  window 2 (1D) / 2x2 (2D), stride 2: x <- x + rho^stride(x) (2D: then
 *         + rho^(stride*pitch)); the stride doubles and the map halves (floor).
 *   GAP   global pooling: rotate-and-sum by stride, 2 stride, .. < dist; block start m
 *         then holds the channel's sum (needs zeros outside the map: follows QUAD).
 *   FC    w = float64[c_out][c] on GAP output, c_out <= cbar, optional bias
 *         float64[c_out]; logit o lands at slot o*dist of the single output ciphertext.
 * Every plaintext multiplied into a ciphertext at level l is encoded at scale q_l with the
 * limbs of level l only, so slot values keep their scale through each rescale. */
#define HEAR_CNN_CONV 1
#define HEAR_CNN_QUAD 2
#define HEAR_CNN_POOL 3
#define HEAR_CNN_GAP 4
#define HEAR_CNN_FC 5
#define HEAR_CNN_BN_QUAD 6
#define HEAR_CNN_AVGPOOL 7
#define HEAR_CNN_GAVGPOOL 8
#define HEAR_STRATEGY_HYBRID 0
#define HEAR_STRATEGY_FULL 1
#define HEAR_STRATEGY_BABY 2
#define HEAR_STRATEGY_GIANT 3
typedef struct hear_cnn_input {
    uint32_t conv_dims;   /* 1 or 2                                                     */
    uint32_t c_in;        /* channels of the input map                                  */
    uint32_t h, w;        /* map size (1D: h = 1)                                       */
    uint32_t pitch;       /* row pitch in slots (0 = w)                                 */
    uint32_t stride;      /* puncture of the input (1 for an encrypted input tensor)    */
    uint32_t level;       /* level of the input ciphertexts (0 = the top level)          */
} hear_cnn_input;
typedef struct hear_cnn_layer {
    uint32_t kind;
    uint32_t c_out;             /* CONV, FC                                             */
    uint32_t f_h, f_w;          /* CONV                                                 */
    const double *w;            /* CONV, FC                                             */
    const double *bias;         /* FC (or NULL)                                         */
    const double *a, *b, *c;    /* QUAD                                                 */
    uint32_t fast;              /* CONV                                                 */
    uint32_t strategy, n1;      /* CONV, FC (n1: HYBRID; 0 = min(4, block shifts))      */
    const double *conv_bias;    /* BN_QUAD (or NULL)                                    */
    const double *bn_gamma, *bn_beta, *bn_mean, *bn_var;   /* BN_QUAD                  */
    double bn_eps;              /* BN_QUAD                                              */
    double act[3];              /* BN_QUAD: act[0] z^2 + act[1] z + act[2]              */
} hear_cnn_layer;
/* The layers become a plan of slot-level operations; every ciphertext of a sample passes
 * through each operation.  Operation kinds: */
#define HEAR_CNN_OP_DIAG 1    /* sum of plaintext (.) rotation products, one rescale    */
#define HEAR_CNN_OP_PACK 2    /* fast convolution step (i)                               */
#define HEAR_CNN_OP_ROTSUM 3  /* rotate-and-sum (pooling, GAP, fast convolution (iii))   */
#define HEAR_CNN_OP_QUAD 4
#define HEAR_CNN_OP_BIAS 5
typedef struct hear_cnn_op_info {
    uint32_t kind;
    uint32_t layer;                 /* index of the layer it comes from                  */
    uint32_t n_in, n_out;           /* ciphertexts per sample before / after             */
    uint32_t level_in, level_out;
    uint32_t n_babies, n_giants;    /* DIAG: rotation amounts (0 included)               */
    uint32_t n_keyswitch;           /* key switches per sample                           */
} hear_cnn_op_info;
hear_status hear_cnn_create(hear_context *ctx, const hear_cnn_input *input, const hear_cnn_layer *layers,
                            size_t n_layers, hear_cnn **out);
void hear_cnn_destroy(hear_cnn *m);
/* Host only (no context, no GPU): the doubles the collapse of the layer list produces, in
 * layer order -- each CONV's weights [c_out][c_in][f_h][f_w], each QUAD's A[c], B[c], C[c]
 * (BN_QUAD layers after collapsing), the FC's weights [c_out][c] -- for auditing the
 * collapse against the trained network. */
hear_status hear_cnn_collapse(const hear_cnn_input *input, const hear_cnn_layer *layers, size_t n_layers,
                              double *out, size_t cap, size_t *n);
/* rotation steps (slots, in [1, N/2)) the plan needs keys for */
hear_status hear_cnn_rotations(const hear_cnn *m, int32_t *steps, size_t cap, size_t *n);
hear_status hear_cnn_ops(const hear_cnn *m, hear_cnn_op_info *ops, size_t cap, size_t *n);
/* slots of the logits in the output ciphertext (FC last), else empty */
hear_status hear_cnn_output_slots(const hear_cnn *m, uint32_t *slots, size_t cap, size_t *n);
/* encrypt one input tensor x = float64[c_in][h][w] (stride-1 input) into the plan's input
 * ciphertexts (ct ids ct_id, ct_id+1, ..; one per input ciphertext); out[n_in] */
hear_status hear_cnn_encrypt(hear_context *ctx, const hear_public_key *pk, const hear_cnn *m, const double *x,
                             uint64_t seed, uint64_t ct_id, hear_ciphertext **out, void *stream);
/* run operations [op0, op1) on n_samples samples: in[s * n_in + i] (n_in of op0, all at
 * op0's input level and one scale), out[s * n_out + j] (n_out of op1-1) */
hear_status hear_cnn_evaluate(const hear_cnn *m, const hear_eval_keys *evk, size_t op0, size_t op1,
                              hear_ciphertext *const *in, size_t n_samples, hear_ciphertext **out, void *stream);

/* ---- slot-batched evaluation (one clip per slot) ----
 * A throughput form of the FC / x^2 networks of hear_model_create for batches of up to N/2
 * clips: slot c of every ciphertext belongs to clip c and ciphertext i of a batch holds
 * feature i of every clip.  An FC layer y = W x is then y_o = rescale(sum_i [w_oi] x_i) with
 * plaintext scalars [w] = round(w q_l) (exact, ties away from zero: the encoding of the
 * constant slot vector w at scale q_l; Methods, "Non-convolutional layers") and no rotation;
 * x^2 is a ciphertext product with relinearisation and rescale; FC_SQ_FC sums the degree-2
 * products y_r u_(c,r) (u = (W2[c,r] W1[r]) x) before one relinearisation and rescale per
 * output.  Only the relinearisation key is needed.  A batch is one contiguous device array
 * [n_ct][2][level+1][N] (NTT domain).  Layers: FC (d_in <= 2^19, no bias), SQUARE,
 * FC_SQ_FC; d_in of the first layer = the batch's ciphertext count. */
hear_status hear_simd_model_create(hear_context *ctx, const hear_layer_desc *layers, size_t n_layers,
                                   uint32_t level, hear_simd_model **out);   /* level 0 = the top level */
hear_status hear_simd_model_info(const hear_simd_model *m, uint32_t *d_in, uint32_t *d_out, uint32_t *level_in,
                                 uint32_t *level_out);
void hear_simd_model_destroy(hear_simd_model *m);
/* x: n_clips x n_features row-major (1 <= n_clips <= N/2); ciphertext i encrypts the slot
 * vector (x[0][i], .., x[n_clips-1][i], 0, ..) at `scale` (0 = the context's default) with
 * randomness stream i of `seed`, then keeps the limbs of `level` (0 = the top level) */
hear_status hear_simd_encrypt(hear_context *ctx, const hear_public_key *pk, const double *x, size_t n_clips,
                              size_t n_features, double scale, uint64_t seed, uint32_t level,
                              hear_simd_batch **out, void *stream);
hear_status hear_simd_batch_info(const hear_simd_batch *b, uint32_t *n_ct, uint32_t *level, double *scale);
/* coefficient domain uint64[n_ct][2][level+1][N] */
hear_status hear_simd_batch_export(const hear_simd_batch *b, uint64_t *out, size_t cap, size_t *n);
hear_status hear_simd_batch_import(hear_context *ctx, const uint64_t *words, size_t n_ct, uint32_t level,
                                   double scale, hear_simd_batch **out, void *stream);
void hear_simd_batch_destroy(hear_simd_batch *b);
/* in: d_in ciphertexts at the model's input level -> out: d_out ciphertexts */
hear_status hear_simd_evaluate(const hear_simd_model *m, const hear_eval_keys *evk, const hear_simd_batch *in,
                               hear_simd_batch **out, void *stream);
/* end to end from host buffers: in = uint64[d_in][2][l+1][N] coefficient domain at the
 * model's input level l and `scale` -> out = uint64[d_out][2][level_out+1][N]; both copies
 * are included */
hear_status hear_simd_evaluate_host(const hear_simd_model *m, const hear_eval_keys *evk, const uint64_t *in_words,
                                    double scale, uint64_t *out_words, size_t cap, size_t *n, uint32_t *level_out,
                                    double *scale_out, void *stream);
/* out: n_clips x n_ct row-major, out[c][o] = slot c of ciphertext o */
hear_status hear_simd_decrypt(hear_context *ctx, const hear_secret_key *sk, const hear_simd_batch *b,
                              size_t n_clips, double *out, size_t cap, size_t *n);

/* ---- rescale for callers that cannot allocate device memory ----
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- a process whose device-memory quota is already held by another
 * framework's caching allocator, a real-time loop that must not take the allocator's
 * locks or latency, a host that owns only pageable host memory and a stream.  It divides
 * a ciphertext by its last prime exactly like hear_rescale, from and to HOST arrays in the
 * coefficient domain: in = uint64[n_poly][level+1][N] (in_words words, every residue of
 * limb i below q_i), out = uint64[n_poly][level][N] (capacity out_cap words), with
 * 1 <= level <= L and 1 <= n_poly <= 3.  It allocates nothing: its device working memory
 * is a fixed 16 MiB array (2^21 words) inside the library, which every GPU that loads the
 * library holds until the process exits; it calls no cudaMalloc, cudaFree or allocating
 * library routine.  Errors: in_words != n_poly*(level+1)*N or an unreduced residue ->
 * HEAR_E_FORMAT; out_cap too small -> HEAR_E_INVAL; n_poly*(2*level+1)*N > 2^21 words ->
 * HEAR_E_UNSUPPORTED; a running profiler (hear_profile_begin) or a `stream` that is being
 * captured into a CUDA graph -> HEAR_E_STATE (the call synchronises `stream`); a CUDA
 * error -> HEAR_E_CUDA and the context is poisoned.  The first call on each device looks
 * up the array's device address.  Every call shares the array, which keeps the last call's
 * contents (each call overwrites everything it reads).  Calls that overlapped on the GPU
 * would race on the array, so the library takes a process-wide lock for the call and
 * synchronises `stream` before returning.  The caller's current CUDA device is restored
 * before the call returns. */
hear_status hear_rescale_noalloc(hear_context *ctx, const uint64_t *in, size_t in_words, uint32_t level,
                                 uint32_t n_poly, uint64_t *out, size_t out_cap, void *stream);

/* ---- tracing: CUDA-event stage profiler and launch counter ---- */
/* One entry per stage (kernel name): how many kernel launches it made, their summed
 * device time (CUDA events recorded on the launching stream around each launch) and
 * the algorithmic HBM bytes they move (each residue read or written once). */
typedef struct hear_profile_entry {
    char name[48];
    uint64_t launches;
    double total_ms;
    double bytes;
} hear_profile_entry;
/* start recording every launch of this context (clears earlier records) */
hear_status hear_profile_begin(hear_context *ctx);
/* wait for the recorded launches, aggregate them per stage and stop recording */
hear_status hear_profile_end(hear_context *ctx, hear_profile_entry *out, size_t cap, size_t *n);
/* kernel launches issued by the library (all contexts) since it was loaded */
uint64_t hear_launch_count(void);
/* kernel launches captured into CUDA graphs with programmatic dependent launch (the
 * kernel may be scheduled while the one before it drains and waits on it on the device:
 * every capture whose pending dependencies are all kernel nodes; HEAR_PDL=0 in the
 * environment turns it off) since the library was loaded */
uint64_t hear_pdl_launch_count(void);

/* ---- NTT launch variants and their tuner ----
 * The forward / inverse NTT has four launch forms with bit-identical results:
 * HEAR_NTT_WIDE (two passes, 4096-word shared-memory tiles, 256 threads), HEAR_NTT_NARROW
 * (two passes, 1024-word tiles, 64 threads: more CTAs for launches of few limbs),
 * HEAR_NTT_FUSED (one launch; a cluster of 8 CTAs per limb exchanges the intermediate
 * through distributed shared memory, so each residue crosses HBM once) and HEAR_NTT_TINY
 * (two passes, 1024-word tiles, 256 threads with radix-4 units: four times the threads of
 * the narrow form for launches of few limbs).  hear_ntt_tune times all four for launches of 1, 2, 4, .. max_limbs limbs in both directions on the
 * context's stream (each timing a replayed CUDA graph of back-to-back transforms) and keeps
 * the fastest two-pass form per power-of-two bucket (larger launches use the largest tuned
 * bucket's choice); the one-launch form is timed but not chosen, because inside whole
 * evaluations it lost clearly where isolated replays sometimes favoured it (a pinned table
 * or hear_ntt_set_variant still selects it).  hear_context_create runs it once (max_limbs 1024, a few
 * tens of milliseconds) unless the environment sets HEAR_NTT_TUNE=0, which keeps a fixed
 * rule (narrow below two wide CTAs per SM, wide above).  It must
 * not run concurrently with other work on the context.  ms_out (optional) receives
 * float[2][16][4] = [forward, inverse][bucket][variant] milliseconds per launch, choice_out
 * (optional) uint8_t[2][16].  hear_ntt_set_variant forces one variant (-1 = back to the
 * table); it exists for tests and measurements. */
#define HEAR_NTT_WIDE 0
#define HEAR_NTT_NARROW 1
#define HEAR_NTT_FUSED 2
#define HEAR_NTT_TINY 3
hear_status hear_ntt_tune(hear_context *ctx, uint32_t max_limbs, int iters, uint8_t *choice_out, float *ms_out);
hear_status hear_ntt_set_variant(hear_context *ctx, int variant);
/* the variant table uint8_t[2][16] ([forward, inverse][bucket]); setting it pins the choice
 * (e.g. to profile a run with the table another run tuned).  The environment variable
 * HEAR_NTT_TABLE (32 digits, forward buckets then inverse) pins it at context creation
 * instead of tuning. */
hear_status hear_ntt_get_table(const hear_context *ctx, uint8_t *table);
hear_status hear_ntt_set_table(hear_context *ctx, const uint8_t *table);

/* ---- key-switch inner product / BSGS inner-sum launch forms (autotuner) ----
 * Three tables of launch forms, each indexed by the log2 bucket (1, 2-3, 4-7, .., 128+) of
 * the batch, all forms bit-identical:
 *   [0] k_ks_inner by ciphertexts per job: 0 = registers capped for 3 CTAs per SM, every
 *       ciphertext in one thread (keys read once per coefficient); 1 = capped for 2 CTAs
 *       (no register spills); 2 / 3 = forms 0 / 1 with the ciphertexts in chunks of 4 over
 *       the grid (more CTAs, keys read once per chunk);
 *   [1] k_ks_inner_rj (one ciphertext, its digits shared by all jobs) by jobs: 0 = 4 jobs
 *       per thread, 1 = 2, 2 = 8; 3 / 4 = 4 / 8 jobs per CTA with each job's key planes
 *       streamed into shared memory by 1-D bulk asynchronous copies (the TMA engine,
 *       double-buffered over the jobs, completion on mbarriers with bounded waits: see
 *       hear_async_status);
 *   [2] k_lincomb by ciphertexts: 0 = 4 giant-step accumulators per pass over the babies,
 *       1 = 8 (registers of 2 CTAs per SM), 2 = 2, 3 = 1 (more passes over the babies,
 *       more chunks of giant steps to spread over the warps), 4 = the baby steps split over
 *       the 8 warps of a CTA, every polynomial of the batch in one thread and the partial
 *       sums added in shared memory (up to 4 ciphertexts; more take form 0).
 * Every table starts at form 0.  hear_ks_tune times every form at the top level on
 * synthetic operands (inner products over 8 jobs for 1, 2, 4, .. max_ct ciphertexts, at
 * most 64; shared-digit products for 2 .. 16 jobs; inner sums with 32 x 4 baby / giant
 * steps up to 4 ciphertexts, 8 x 8 above) as replayed CUDA graphs of `iters` launches and keeps the fastest per bucket
 * (larger buckets take the largest tuned bucket's form).  It allocates up to a few GB of
 * scratch for the large parameter sets and must not run concurrently with other work on
 * the context.  choice_out (optional): uint8_t[3][8]; ms_out (optional): float[3][8][8]
 * milliseconds per launch (0 = not timed).  hear_ks_set_variant forces form v (0..7) in every
 * table (taken modulo the table's form count; -1 = back to the tables), for tests and
 * measurements.  The table can be read and pinned (uint8_t[3][8]); the environment
 * variable HEAR_KS_TABLE (24 digits) pins it at context creation. */
hear_status hear_ks_tune(hear_context *ctx, uint32_t max_ct, int iters, uint8_t *choice_out, float *ms_out);
hear_status hear_ks_get_table(const hear_context *ctx, uint8_t *table);
hear_status hear_ks_set_table(hear_context *ctx, const uint8_t *table);
hear_status hear_ks_set_variant(hear_context *ctx, int variant);

/* ---- bounded device waits ----
 * Kernels that wait on the device (the bulk-copy key inner products wait on shared-memory
 * mbarriers for their copies) give up after about a second of SM cycles: the CTA counts the
 * timeout in a process-wide device counter, lets its copies in flight land and returns, its
 * outputs left unwritten.  hear_async_status synchronises the context's default stream,
 * reads and clears that counter of the context's device: HEAR_OK if no wait ran out,
 * HEAR_E_TIMEOUT (and *timeouts = how many, optional) if some did -- results computed since
 * the last check are then not to be trusted.  The context stays usable either way.  No
 * device fault or hang is involved: a wait that runs out is an ordinary return. */
hear_status hear_async_status(hear_context *ctx, uint32_t *timeouts);
/* debug: one CTA waits on an mbarrier that nothing completes, with a limit of limit_cycles SM
 * cycles (>= 0), on the context's default stream; *timed_out = 1 when the wait ran out (it
 * is then counted for hear_async_status like any other), 0 when it completed.  Tests the
 * bounded-wait path without a fault. */
hear_status hear_dbg_wait_probe(hear_context *ctx, long long limit_cycles, uint32_t *timed_out);

/* ---- debug: ring products through the NTT kernels (tests only) ---- */
/* out = a * b in Z_q[X]/(X^N+1) for limb prime index `prime` (0..n_q+n_p-1), coefficient domain */
/* the plaintext scalar of weight w at scale q (q a prime of the chain or any q < 2^62):
 * round(w q) computed exactly, ties away from zero -- the coefficient the slot-batched FC
 * layers multiply by.  Host only (no device needed).  HEAR_E_INVAL for a non-finite w or
 * |w q| >= 2^62. */
hear_status hear_dbg_round_scalar(double w, uint64_t q, int64_t *out);
/* lane operations per second of an integer multiply-add form (kind 0: mad.wide.u32 --
 * 32 x 32 -> 64 bits plus a 64-bit addend, the step of the slot-batched matrix product;
 * kind 1: mad.lo.u32), from a throughput kernel of 8 independent chains per thread on every
 * SM (iters multiply-adds per chain, iters in [1, 2^20]); the roofline denominator of the
 * integer-multiply-bound kernels */
hear_status hear_dbg_imad_peak(hear_context *ctx, int kind, uint32_t iters, double *lane_ops_per_s);
/* butterflies per second of the NTT's own arithmetic with no memory traffic: every thread
 * keeps one radix-16 unit and its twiddles in registers and applies the unit's four stages
 * iters times (iters in [1, 2^20]) -- the forward butterfly (inverse = 0: Shoup product,
 * Harvey lazy add / subtract, the 2q correction for primes of 58 bits and more) or the
 * inverse one -- on every SM, warp w on prime w mod (n_q + n_p).  The measured ceiling of
 * the transforms' butterfly rate on the integer pipes (their roofline denominator). */
hear_status hear_dbg_bfly_peak(hear_context *ctx, int inverse, uint32_t iters, double *butterflies_per_s);
hear_status hear_dbg_poly_mul(hear_context *ctx, uint32_t prime, const uint64_t *a, const uint64_t *b,
                              uint64_t *out);
/* forward+inverse NTT round trip of n_limb limbs (prime i % (n_q+n_p)) in place */
hear_status hear_dbg_ntt_roundtrip(hear_context *ctx, uint64_t *limbs, size_t n_limb);
/* device time of one forward and one inverse NTT over n_limb limbs of zero data (limb i
 * uses prime i % (n_q+n_p)), averaged over `iters` launches after one warm-up; for tuning */
hear_status hear_dbg_ntt_time(hear_context *ctx, size_t n_limb, int iters, float *ms_fwd, float *ms_inv);

#ifdef __cplusplus
}
#endif
#endif
