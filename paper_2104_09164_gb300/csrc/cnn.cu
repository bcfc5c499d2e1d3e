// cnn.cu -- the encrypted skeleton CNN: plan construction (multi-channel and fast
// homomorphic convolution, pooling by rotate-and-sum, FC on pooled features, per-channel
// quadratic activation) and batched evaluation of the plan on the GPU.
//
// Every operation runs on the ciphertexts of all samples at once: a batch is laid out
// [n_ct][C][2][level+1][N] (ciphertext index of the sample outermost, samples contiguous),
// so the hoisted rotations of input ciphertext i cover every sample in one key switch
// launch and the plaintext products read each plaintext once for all samples.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>
#include "cnn.h"

namespace hear {
namespace {

int32_t wrap(int64_t a, uint32_t S) {
    int64_t r = a % (int64_t)S;
    if (r < 0) r += S;
    return (int32_t)r;
}

uint32_t pow2_at_least(uint64_t v) {
    uint32_t p = 1;
    while (p < v) p *= 2;
    return p;
}

DevBuf upload_bytes(const void *host, size_t bytes, cudaStream_t st) {
    DevBuf b(bytes, st);
    HEAR_CHECK_CUDA(cudaMemcpyAsync(b.p, host, bytes, cudaMemcpyHostToDevice, st));
    return b;
}

// Slot geometry of the feature maps one sample's ciphertexts carry.
struct Geo {
    uint32_t S = 0, dist = 0, cbar = 0;
    uint32_t h = 0, w = 0, pitch = 0, stride = 1;
    uint32_t n_ct = 0, lr = 0, channels = 0;
    uint32_t kind = 0;            // 0: ct i block m = channel cbar*i + m; 1: copies m mod c; 2: packed
    uint32_t n_p = 1;             // packed: phases per ciphertext
    std::vector<int32_t> offs{0}; // phase offsets (slots)
    bool clean = true;            // non-valid slots hold zeros
    bool pooled = false;          // after GAP: channel sums at block starts
    uint32_t chan(uint32_t i, uint32_t m, uint32_t p) const {
        if (kind == 1) return m % channels;
        if (kind == 2) return cbar * (i * n_p + p) + m;
        return cbar * i + m;
    }
    struct Pos {
        int32_t y, x;
        uint32_t off;
    };
    std::vector<Pos> positions() const {
        std::vector<Pos> v;
        for (uint32_t y = 0; y < h; y++)
            for (uint32_t x = 0; x < w; x++) v.push_back(Pos{(int32_t)y, (int32_t)x, stride * (y * pitch + x)});
        return v;
    }
};

// a = r + dist*l  ->  (hoisted baby step b, giant step g)
void split_rot(uint32_t strategy, uint32_t n1, int64_t r, uint32_t l, uint32_t dist, int64_t &b, int64_t &g) {
    switch (strategy) {
        case HEAR_STRATEGY_FULL: b = r + (int64_t)dist * l; g = 0; break;
        case HEAR_STRATEGY_BABY: b = r; g = (int64_t)dist * l; break;
        case HEAR_STRATEGY_GIANT: b = (int64_t)dist * l; g = r; break;
        case HEAR_STRATEGY_HYBRID: b = r + (int64_t)dist * (l % n1); g = (int64_t)dist * n1 * (l / n1); break;
        default: throw Error(HEAR_E_INVAL, "unknown strategy");
    }
}

// Host slot vectors -> plaintexts [count][level+1][N] at dst (NTT domain; Montgomery form
// when `mont`), encoded at per-vector scales.
void encode_into(hear_context *c, const double *z, size_t count, const double *scales, uint32_t level, bool mont,
                 uint64_t *dst, cudaStream_t st) {
    if (!count) return;
    const uint32_t n = c->n, L1 = level + 1;
    std::vector<int64_t> m(count * n);
    encode_many(*encoder(c), z, count, scales, m.data());
    DevBuf dm = upload_bytes(m.data(), m.size() * 8, st);
    i64_to_limbs_batch(c, (const int64_t *)dm.p, dst, (uint32_t)count, level, st);
    ntt_forward(c, dst, (uint32_t)count * L1, map_q(level, c->n_q), st);
    if (mont) to_mont(c, dst, (uint32_t)count * L1, map_q(level, c->n_q), st);
    HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
}

// Dense diagonal operation: out_j = sum_g rho^g(sum_(b,i) pt[g][j][b][i] (.) rho^b(x_i)).
// `raw` lists (b, g, source) for every contribution; fill(j, i, source, z) adds the slot
// vector of that contribution from input i to output j into z.
template <class Fill>
void build_diag(hear_context *c, hear_cnn::Op &op, const std::vector<std::tuple<int32_t, int32_t, uint64_t>> &raw,
                Fill fill, cudaStream_t st) {
    const uint32_t S = c->n / 2, L1 = op.level_in + 1;
    std::set<int32_t> bs{0}, gs{0};
    for (auto &t : raw) {
        bs.insert(std::get<0>(t));
        gs.insert(std::get<1>(t));
    }
    op.babies.assign(bs.begin(), bs.end());
    op.giants.assign(gs.begin(), gs.end());
    const uint32_t nb = (uint32_t)op.babies.size(), ng = (uint32_t)op.giants.size();
    std::map<std::pair<uint32_t, uint32_t>, std::vector<uint64_t>> src;
    for (auto &t : raw) {
        uint32_t bi = (uint32_t)(std::lower_bound(op.babies.begin(), op.babies.end(), std::get<0>(t)) - op.babies.begin());
        uint32_t gi = (uint32_t)(std::lower_bound(op.giants.begin(), op.giants.end(), std::get<1>(t)) - op.giants.begin());
        src[{bi, gi}].push_back(std::get<2>(t));
    }
    const uint64_t plane = (uint64_t)L1 * c->n;
    const size_t n_pt = (size_t)ng * op.n_out * nb * op.n_in;
    op.pts = DevBuf(n_pt * plane * 8, nullptr);
    const double ql = (double)c->primes[op.level_in];
    const size_t chunk = std::max<size_t>(1, std::min<size_t>(256, (64u << 20) / (S * 8)));
    std::vector<double> z, zr;
    std::vector<double> scales;
    for (size_t q0 = 0; q0 < n_pt; q0 += chunk) {
        const size_t cnt = std::min(chunk, n_pt - q0);
        zr.assign(cnt * S, 0.0);
        scales.assign(cnt, ql);
        for (size_t k = 0; k < cnt; k++) {
            size_t q = q0 + k;
            const uint32_t i = (uint32_t)(q % op.n_in);
            const uint32_t bi = (uint32_t)((q / op.n_in) % nb);
            const uint32_t j = (uint32_t)((q / ((size_t)op.n_in * nb)) % op.n_out);
            const uint32_t gi = (uint32_t)(q / ((size_t)op.n_in * nb * op.n_out));
            auto it = src.find({bi, gi});
            if (it == src.end()) continue;
            z.assign(S, 0.0);
            for (uint64_t s : it->second) fill(j, i, s, z.data());
            // pre-rotate by rho^(-g): entry t takes z[t - g]
            const uint32_t g = (uint32_t)op.giants[gi];
            double *d = &zr[k * S];
            for (uint32_t t = 0; t < S; t++) d[t] = z[(t + S - g) % S];
        }
        encode_into(c, zr.data(), cnt, scales.data(), op.level_in, true, op.pts.u64() + q0 * plane, st);
    }
}

const uint64_t *need_key(const hear_eval_keys *evk, uint32_t g) {
    const uint64_t *k = evk->key(g);
    HEAR_REQUIRE(k, HEAR_E_NOKEY, "missing switching key for galois element " + std::to_string(g));
    return k;
}

std::vector<Rot> rots_for(const hear_context *c, const hear_eval_keys *evk, const std::vector<int32_t> &steps) {
    std::vector<Rot> r;
    for (int32_t s : steps) {
        uint32_t g = galois_of(c, s);
        r.push_back(Rot{need_key(evk, g), g});
    }
    return r;
}

// Layer collapsing (Methods, "Non-convolutional layers"): a block's convolution bias, batch
// normalisation and quadratic activation become one quadratic per feature map, and the
// 1/2 (1D) or 1/4 (2D) of each average pooling and the 1/(h*w) of the global average
// pooling move into the weights of the next linear layer, so that pooling is a plain sum.
// With BN(y + bias) = s*y + t, s = gamma / sqrt(var + eps), t = s*(bias - mean) + beta and
// the activation a*z^2 + b*z + c:  A = a*s^2, B = 2*a*s*t + b*s, C = a*t^2 + b*t + c.
// The doubles are formed in exactly the order written here (A = (a*s)*s,
// B = ((2*a)*s)*t + b*s, C = ((a*t)*t + b*t) + c; conv weights w*scale, FC weights
// (w*scale)/(h*w)), so every encoded plaintext is reproducible from the description.
// Layers that are already collapsed pass through unchanged.
struct Collapsed {
    std::vector<hear_cnn_layer> layers;
    std::vector<std::unique_ptr<std::vector<double>>> store;
    const double *keep(std::vector<double> &&v) {
        store.push_back(std::make_unique<std::vector<double>>(std::move(v)));
        return store.back()->data();
    }
};

Collapsed collapse_layers(const hear_cnn_input *in, const hear_cnn_layer *layers, size_t n_layers) {
    Collapsed out;
    const uint32_t dims = in->conv_dims;
    uint32_t h = in->h, w = in->w, channels = in->c_in;
    double scale = 1.0;        // pending average-pooling factor for the next linear layer
    double divisor = 1.0;      // pending global-average-pooling divisor (h*w) for the FC
    for (size_t li = 0; li < n_layers; li++) {
        hear_cnn_layer d = layers[li];
        if (d.kind == HEAR_CNN_CONV) {
            HEAR_REQUIRE(d.w && d.c_out && d.f_h && d.f_w, HEAR_E_INVAL, "conv needs weights and filter sizes");
            if (scale != 1.0) {
                const size_t nw = (size_t)d.c_out * channels * d.f_h * d.f_w;
                std::vector<double> v(nw);
                for (size_t i = 0; i < nw; i++) v[i] = d.w[i] * scale;
                d.w = out.keep(std::move(v));
            }
            scale = 1.0;
            channels = d.c_out;
        } else if (d.kind == HEAR_CNN_BN_QUAD) {
            HEAR_REQUIRE(d.bn_gamma && d.bn_beta && d.bn_mean && d.bn_var, HEAR_E_INVAL,
                         "batch normalisation needs gamma, beta, mean and var");
            HEAR_REQUIRE(d.bn_eps >= 0.0, HEAR_E_INVAL, "batch-normalisation epsilon must be >= 0");
            std::vector<double> A(channels), B(channels), C(channels);
            const double a = d.act[0], b = d.act[1], cc = d.act[2];
            for (uint32_t k = 0; k < channels; k++) {
                HEAR_REQUIRE(d.bn_var[k] + d.bn_eps > 0.0, HEAR_E_INVAL, "batch-normalisation variance must be > 0");
                const double sk = d.bn_gamma[k] / std::sqrt(d.bn_var[k] + d.bn_eps);
                const double bias = d.conv_bias ? d.conv_bias[k] : 0.0;
                const double tk = sk * (bias - d.bn_mean[k]) + d.bn_beta[k];
                A[k] = a * sk * sk;
                B[k] = 2.0 * a * sk * tk + b * sk;
                C[k] = a * tk * tk + b * tk + cc;
            }
            hear_cnn_layer q{};
            q.kind = HEAR_CNN_QUAD;
            q.a = out.keep(std::move(A));
            q.b = out.keep(std::move(B));
            q.c = out.keep(std::move(C));
            d = q;
        } else if (d.kind == HEAR_CNN_AVGPOOL || d.kind == HEAR_CNN_POOL) {
            if (d.kind == HEAR_CNN_AVGPOOL) scale *= dims == 1 ? 0.5 : 0.25;
            d.kind = HEAR_CNN_POOL;
            w /= 2;
            if (dims == 2) h /= 2;
        } else if (d.kind == HEAR_CNN_GAVGPOOL || d.kind == HEAR_CNN_GAP) {
            if (d.kind == HEAR_CNN_GAVGPOOL) {
                HEAR_REQUIRE(h >= 1 && w >= 1, HEAR_E_INVAL, "pooling an empty map");
                divisor = (double)(h * w);
            }
            d.kind = HEAR_CNN_GAP;
        } else if (d.kind == HEAR_CNN_FC) {
            HEAR_REQUIRE(d.w && d.c_out, HEAR_E_INVAL, "FC needs weights");
            if (scale != 1.0 || divisor != 1.0) {
                const size_t nw = (size_t)d.c_out * channels;
                std::vector<double> v(nw);
                for (size_t i = 0; i < nw; i++) v[i] = (d.w[i] * scale) / divisor;
                d.w = out.keep(std::move(v));
            }
            scale = divisor = 1.0;
        } else {
            HEAR_REQUIRE(d.kind == HEAR_CNN_QUAD, HEAR_E_INVAL, "unknown layer kind");
        }
        out.layers.push_back(d);
    }
    return out;
}

}  // namespace

hear_cnn *cnn_create(hear_context *c, const hear_cnn_input *in, const hear_cnn_layer *layers_in, size_t n_layers) {
    HEAR_REQUIRE(in && layers_in && n_layers, HEAR_E_INVAL, "no layers");
    HEAR_REQUIRE(in->conv_dims == 1 || in->conv_dims == 2, HEAR_E_INVAL, "conv_dims must be 1 or 2");
    const Collapsed collapsed = collapse_layers(in, layers_in, n_layers);
    const hear_cnn_layer *layers = collapsed.layers.data();
    HEAR_REQUIRE(in->conv_dims == 1 || in->conv_dims == 2, HEAR_E_INVAL, "conv_dims must be 1 or 2");
    HEAR_REQUIRE(in->c_in && in->h && in->w && in->stride, HEAR_E_INVAL, "empty input map");
    HEAR_REQUIRE(in->conv_dims == 2 || in->h == 1, HEAR_E_INVAL, "1D maps have h = 1");
    cudaStream_t st = c->stream;
    auto m = std::make_unique<hear_cnn>();
    m->ctx = c;
    const uint32_t S = c->n / 2, dims = in->conv_dims;
    Geo g;
    g.S = S;
    g.h = in->h;
    g.w = in->w;
    g.pitch = in->pitch ? in->pitch : in->w;
    HEAR_REQUIRE(g.pitch >= g.w, HEAR_E_INVAL, "pitch must be >= w");
    g.stride = in->stride;
    g.dist = pow2_at_least((uint64_t)g.stride * g.h * g.pitch);
    HEAR_REQUIRE(g.dist <= S, HEAR_E_UNSUPPORTED, "input map does not fit a ciphertext");
    g.cbar = S / g.dist;
    g.channels = in->c_in;
    if (in->c_in < g.cbar) {
        HEAR_REQUIRE(g.cbar % in->c_in == 0, HEAR_E_INVAL, "channel copies must fill the blocks");
        g.kind = 1;
        g.n_ct = 1;
        g.lr = in->c_in;
    } else {
        HEAR_REQUIRE(in->c_in % g.cbar == 0, HEAR_E_INVAL, "channels must fill whole ciphertexts");
        g.kind = 0;
        g.n_ct = in->c_in / g.cbar;
        g.lr = g.cbar;
    }
    m->in_kind = g.kind;
    m->in_c = in->c_in;
    m->in_dist = g.dist;
    m->in_h = g.h;
    m->in_w = g.w;
    m->in_pitch = g.pitch;
    HEAR_REQUIRE(in->level <= c->L, HEAR_E_LEVEL, "input level above the top level");
    uint32_t level = in->level ? in->level : c->L;
    std::set<int32_t> rots;
    auto push = [&](hear_cnn::Op &&op, uint32_t layer) {
        op.level_out = level;
        for (int32_t b : op.babies)
            if (b) rots.insert(b);
        for (int32_t gg : op.giants)
            if (gg) rots.insert(gg);
        for (int32_t o : op.offs)
            if (o) rots.insert(wrap(-(int64_t)o, S));
        for (int32_t s : op.steps) rots.insert(s);
        m->ops.push_back(std::move(op));
        m->op_layer.push_back(layer);
    };
    for (size_t li = 0; li < n_layers; li++) {
        const hear_cnn_layer &d = layers[li];
        HEAR_REQUIRE(!g.pooled || d.kind == HEAR_CNN_FC, HEAR_E_INVAL, "only FC may follow global pooling");
        if (d.kind == HEAR_CNN_CONV) {
            HEAR_REQUIRE(d.w && d.c_out && d.f_h && d.f_w && (d.f_h % 2) && (d.f_w % 2), HEAR_E_INVAL,
                         "conv needs weights and odd filter sizes");
            HEAR_REQUIRE(dims == 2 || d.f_h == 1, HEAR_E_INVAL, "1D convolution has f_h = 1");
            HEAR_REQUIRE(d.c_out % g.cbar == 0, HEAR_E_INVAL, "c_out must be a multiple of the channels per ciphertext");
            const uint32_t c_in = g.channels, fh = d.f_h, fw = d.f_w;
            if (d.fast) {
                HEAR_REQUIRE(g.stride > 1 && g.kind == 0, HEAR_E_INVAL, "fast convolution needs a punctured input");
                HEAR_REQUIRE(level >= 2, HEAR_E_LEVEL, "not enough levels for the network");
                uint32_t n_p = dims == 1 ? g.stride : g.stride * g.stride;
                while (g.n_ct % n_p) n_p /= 2;
                const uint32_t nx = std::min(g.stride, n_p), ny = n_p / nx;
                hear_cnn::Op op;
                op.kind = hear_cnn::kPack;
                op.n_in = g.n_ct;
                op.n_out = g.n_ct / n_p;
                op.level_in = level;
                for (uint32_t py = 0; py < ny; py++)
                    for (uint32_t px = 0; px < nx; px++) op.offs.push_back((int32_t)(py * g.pitch + px));
                std::vector<double> mask(S, 0.0);
                for (auto &p : g.positions())
                    for (uint32_t mb = 0; mb < g.cbar; mb++) mask[(size_t)mb * g.dist + p.off] = 1.0;
                op.mask = DevBuf((size_t)(level + 1) * c->n * 8, nullptr);
                const double ql = (double)c->primes[level];
                encode_into(c, mask.data(), 1, &ql, level, true, op.mask.u64(), st);
                level -= 1;
                push(std::move(op), (uint32_t)li);
                g.kind = 2;
                g.n_p = n_p;
                g.n_ct /= n_p;
                g.offs = m->ops.back().offs;
                g.lr = g.cbar;
            }
            HEAR_REQUIRE(level >= 1, HEAR_E_LEVEL, "not enough levels for the network");
            hear_cnn::Op op;
            op.kind = hear_cnn::kDiag;
            op.n_in = g.n_ct;
            op.n_out = d.c_out / g.cbar;
            op.level_in = level;
            const uint32_t strategy = d.strategy;
            const uint32_t n1 = d.n1 ? d.n1 : std::min(4u, g.lr);
            HEAR_REQUIRE(n1 >= 1, HEAR_E_INVAL, "n1 must be positive");
            // rotation of tap (u, v), block shift l: r + dist*l; source id = (tap, l)
            std::vector<std::tuple<int32_t, int32_t, uint64_t>> raw;
            for (uint32_t u = 0; u < fh; u++)
                for (uint32_t v = 0; v < fw; v++) {
                    const int64_t r = (int64_t)g.stride * (((int64_t)u - fh / 2) * g.pitch + ((int64_t)v - fw / 2));
                    for (uint32_t l = 0; l < g.lr; l++) {
                        int64_t b, gg;
                        split_rot(strategy, n1, r, l, g.dist, b, gg);
                        raw.emplace_back(wrap(b, S), wrap(gg, S), ((uint64_t)(u * fw + v) << 32) | l);
                    }
                }
            const Geo gin = g;
            const auto pos = gin.positions();
            const double *W = d.w;
            auto fill = [&](uint32_t j, uint32_t i, uint64_t s, double *z) {
                const uint32_t tap = (uint32_t)(s >> 32), l = (uint32_t)(s & 0xffffffffu);
                const int32_t du = (int32_t)(tap / fw) - (int32_t)(fh / 2), dv = (int32_t)(tap % fw) - (int32_t)(fw / 2);
                for (uint32_t mb = 0; mb < gin.cbar; mb++) {
                    const uint32_t o = gin.cbar * j + mb;
                    for (uint32_t p = 0; p < gin.offs.size(); p++) {
                        const uint32_t ch = gin.chan(i, (mb + l) % gin.cbar, p);
                        const double wv = W[(((size_t)o * c_in + ch) * fh + tap / fw) * fw + tap % fw];
                        for (auto &q : pos) {
                            const int32_t yy = q.y + du, xx = q.x + dv;
                            if (yy < 0 || yy >= (int32_t)gin.h || xx < 0 || xx >= (int32_t)gin.w) continue;
                            z[(size_t)mb * gin.dist + q.off + gin.offs[p]] += wv;
                        }
                    }
                }
            };
            build_diag(c, op, raw, fill, st);
            level -= 1;
            push(std::move(op), (uint32_t)li);
            if (d.fast) {
                hear_cnn::Op post;
                post.kind = hear_cnn::kRotsum;
                post.n_in = post.n_out = d.c_out / g.cbar;
                post.level_in = level;
                const uint32_t nx = std::min(g.stride, g.n_p), ny = g.n_p / nx;
                for (uint32_t t = 1; t < nx; t *= 2) post.steps.push_back((int32_t)t);
                for (uint32_t t = 1; t < ny; t *= 2) post.steps.push_back((int32_t)(t * g.pitch));
                push(std::move(post), (uint32_t)li);
            }
            g.kind = 0;
            g.n_p = 1;
            g.offs = {0};
            g.n_ct = d.c_out / g.cbar;
            g.lr = g.cbar;
            g.channels = d.c_out;
            g.clean = !d.fast;
        } else if (d.kind == HEAR_CNN_QUAD) {
            HEAR_REQUIRE(d.a && d.b && d.c, HEAR_E_INVAL, "quad needs a, b, c");
            HEAR_REQUIRE(level >= 2, HEAR_E_LEVEL, "not enough levels for the network");
            hear_cnn::Op op;
            op.kind = hear_cnn::kQuad;
            op.n_in = op.n_out = g.n_ct;
            op.level_in = level;
            const auto pos = g.positions();
            std::vector<double> A((size_t)g.n_ct * S, 0.0);
            op.B.assign((size_t)g.n_ct * S, 0.0);
            op.C.assign((size_t)g.n_ct * S, 0.0);
            for (uint32_t i = 0; i < g.n_ct; i++)
                for (uint32_t mb = 0; mb < g.cbar; mb++) {
                    const uint32_t ch = g.chan(i, mb, 0);
                    for (auto &q : pos) {
                        const size_t t = (size_t)i * S + (size_t)mb * g.dist + q.off;
                        A[t] = d.a[ch];
                        op.B[t] = d.b[ch];
                        op.C[t] = d.c[ch];
                    }
                }
            op.A = DevBuf((size_t)g.n_ct * (level + 1) * c->n * 8, nullptr);
            std::vector<double> scales(g.n_ct, (double)c->primes[level]);
            encode_into(c, A.data(), g.n_ct, scales.data(), level, true, op.A.u64(), st);
            level -= 2;
            push(std::move(op), (uint32_t)li);
            g.clean = true;
        } else if (d.kind == HEAR_CNN_POOL) {
            hear_cnn::Op op;
            op.kind = hear_cnn::kRotsum;
            op.n_in = op.n_out = g.n_ct;
            op.level_in = level;
            op.steps.push_back((int32_t)g.stride);
            if (dims == 2) op.steps.push_back((int32_t)(g.stride * g.pitch));
            push(std::move(op), (uint32_t)li);
            g.stride *= 2;
            g.w /= 2;
            if (dims == 2) g.h /= 2;
            HEAR_REQUIRE(g.w >= 1 && g.h >= 1, HEAR_E_INVAL, "pooling an empty map");
            g.clean = false;
        } else if (d.kind == HEAR_CNN_GAP) {
            HEAR_REQUIRE(g.clean, HEAR_E_INVAL, "global pooling needs zeros outside the map (place it after QUAD)");
            hear_cnn::Op op;
            op.kind = hear_cnn::kRotsum;
            op.n_in = op.n_out = g.n_ct;
            op.level_in = level;
            for (uint32_t t = g.stride; t < g.dist; t *= 2) op.steps.push_back((int32_t)t);
            push(std::move(op), (uint32_t)li);
            g.pooled = true;
        } else if (d.kind == HEAR_CNN_FC) {
            HEAR_REQUIRE(g.pooled && li + 1 == n_layers, HEAR_E_INVAL, "FC must follow GAP and end the network");
            HEAR_REQUIRE(d.w && d.c_out && d.c_out <= g.cbar, HEAR_E_INVAL, "FC outputs must fit the blocks");
            HEAR_REQUIRE(level >= 1, HEAR_E_LEVEL, "not enough levels for the network");
            hear_cnn::Op op;
            op.kind = hear_cnn::kDiag;
            op.n_in = g.n_ct;
            op.n_out = 1;
            op.level_in = level;
            const uint32_t n1 = d.n1 ? d.n1 : std::min(4u, g.cbar);
            std::vector<std::tuple<int32_t, int32_t, uint64_t>> raw;
            for (uint32_t dl = 0; dl < g.cbar; dl++) {
                int64_t b, gg;
                split_rot(d.strategy, n1, 0, dl, g.dist, b, gg);
                raw.emplace_back(wrap(b, S), wrap(gg, S), dl);
            }
            const Geo gin = g;
            const uint32_t c_feat = g.channels, n_cls = d.c_out;
            const double *W = d.w;
            auto fill = [&](uint32_t, uint32_t i, uint64_t dl, double *z) {
                for (uint32_t o = 0; o < n_cls; o++)
                    z[(size_t)o * gin.dist] += W[(size_t)o * c_feat + gin.chan(i, (uint32_t)((o + dl) % gin.cbar), 0)];
            };
            build_diag(c, op, raw, fill, st);
            level -= 1;
            push(std::move(op), (uint32_t)li);
            if (d.bias) {
                hear_cnn::Op b;
                b.kind = hear_cnn::kBias;
                b.n_in = b.n_out = 1;
                b.level_in = level;
                b.bias.assign(S, 0.0);
                for (uint32_t o = 0; o < n_cls; o++) b.bias[(size_t)o * g.dist] = d.bias[o];
                push(std::move(b), (uint32_t)li);
            }
            for (uint32_t o = 0; o < n_cls; o++) m->out_slots.push_back(o * g.dist);
            g.n_ct = 1;
        } else {
            throw Error(HEAR_E_INVAL, "unknown layer kind");
        }
    }
    m->rotations.assign(rots.begin(), rots.end());
    return m.release();
}

double cnn_scale_after(const hear_cnn *m, size_t op0, size_t op1, double scale) {
    const hear_context *c = m->ctx;
    for (size_t k = op0; k < op1; k++) {
        const hear_cnn::Op &op = m->ops[k];
        const double ql = (double)c->primes[op.level_in];
        if (op.kind == hear_cnn::kDiag || op.kind == hear_cnn::kPack) {
            scale = scale * ql / ql;
        } else if (op.kind == hear_cnn::kQuad) {
            const double su = scale * ql / ql;
            scale = scale * su / (double)c->primes[op.level_in - 1];
        }
    }
    return scale;
}

namespace {
// plaintexts of op k whose scale follows the evaluation's scale (B and C of QUAD, BIAS)
const uint64_t *scaled_pts(const hear_cnn *m, size_t k, double scale, cudaStream_t st) {
    std::lock_guard<std::mutex> g(m->mu);
    auto key = std::make_pair(k, scale);
    auto it = m->scaled.find(key);
    if (it != m->scaled.end()) return it->second.u64();
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HEAR_CHECK_CUDA(cudaStreamIsCapturing(st, &cs));
    HEAR_REQUIRE(cs == cudaStreamCaptureStatusNone, HEAR_E_STATE, "plaintexts for this scale missing during capture");
    hear_context *c = m->ctx;
    const hear_cnn::Op &op = m->ops[k];
    const uint32_t n = c->n, S = n / 2;
    cudaStream_t cs0 = c->stream;
    DevBuf buf;
    if (op.kind == hear_cnn::kQuad) {
        const uint32_t l = op.level_in;
        const double ql = (double)c->primes[l];
        const double su = scale * ql / ql, sv = scale * su / (double)c->primes[l - 1];
        const size_t wb = (size_t)op.n_in * l * n, wc = (size_t)op.n_in * (l - 1) * n;
        buf = DevBuf((wb + wc) * 8, nullptr);
        std::vector<double> s1(op.n_in, su), s2(op.n_in, sv);
        encode_into(c, op.B.data(), op.n_in, s1.data(), l - 1, false, buf.u64(), cs0);
        encode_into(c, op.C.data(), op.n_in, s2.data(), l - 2, false, buf.u64() + wb, cs0);
    } else {
        buf = DevBuf((size_t)(op.level_in + 1) * n * 8, nullptr);
        (void)S;
        encode_into(c, op.bias.data(), 1, &scale, op.level_in, false, buf.u64(), cs0);
    }
    return m->scaled.emplace(key, std::move(buf)).first->second.u64();
}
}  // namespace

DevBuf cnn_evaluate(const hear_cnn *m, const hear_eval_keys *evk, size_t op0, size_t op1, const uint64_t *x,
                    uint32_t C, double scale_in, double *scale_out, cudaStream_t st) {
    hear_context *c = m->ctx;
    const uint32_t n = c->n;
    double scale = scale_in;
    // make every scale-dependent plaintext before the first launch (none inside a capture)
    {
        double s = scale_in;
        for (size_t k = op0; k < op1; k++) {
            const hear_cnn::Op &op = m->ops[k];
            if (op.kind == hear_cnn::kQuad || op.kind == hear_cnn::kBias) scaled_pts(m, k, s, st);
            s = cnn_scale_after(m, k, k + 1, s);
        }
    }
    DevBuf cur;
    const uint64_t *xin = x;
    for (size_t k = op0; k < op1; k++) {
        const hear_cnn::Op &op = m->ops[k];
        const uint32_t level = op.level_in, L1 = level + 1;
        const uint64_t ctw = 2ull * L1 * n;
        DevBuf next;
        if (op.kind == hear_cnn::kDiag) {
            const uint32_t nb = (uint32_t)op.babies.size(), ng = (uint32_t)op.giants.size();
            const uint64_t batch_in = (uint64_t)op.n_in * C * ctw, batch_out = (uint64_t)op.n_out * C * ctw;
            // babies [nb][n_in][C]: slot 0 = the inputs themselves, then the hoisted rotations
            DevBuf babies((size_t)nb * batch_in * 8, st);
            HEAR_CHECK_CUDA(cudaMemcpyAsync(babies.p, xin, batch_in * 8, cudaMemcpyDeviceToDevice, st));
            if (nb > 1) {
                std::vector<int32_t> bs(op.babies.begin() + 1, op.babies.end());
                rotate_hoisted(c, level, op.n_in * C, xin, rots_for(c, evk, bs), babies.u64() + batch_in, st);
            }
            // inner sums G[gi][j] = sum_(b,i) pt (.) baby  (lazy: no rescale yet)
            DevBuf G((size_t)ng * batch_out * 8, st);
            lincomb(c, level, C, nb * op.n_in, ng * op.n_out, babies.u64(), op.pts.u64(), G.u64(), st);
            if (ng > 1) {
                std::vector<int32_t> gsteps;
                for (uint32_t gi = 1; gi < ng; gi++)
                    for (uint32_t j = 0; j < op.n_out; j++) gsteps.push_back(op.giants[gi]);
                DevBuf R((size_t)(ng - 1) * batch_out * 8, st);
                rotate_each(c, level, (ng - 1) * op.n_out, C, G.u64() + batch_out, rots_for(c, evk, gsteps), R.u64(),
                            st);
                sum_add_ct(c, level, 2 * op.n_out * C, R.u64(), batch_out, ng - 1, G.u64(), G.u64(), st);
            }
            next = DevBuf((size_t)op.n_out * C * 2 * level * n * 8, st);
            DevBuf tmp((size_t)op.n_out * C * 2 * level * n * 8, st);
            rescale(c, level, 2 * op.n_out * C, G.u64(), next.u64(), tmp.u64(), st);
            const double ql = (double)c->primes[level];
            scale = scale * ql / ql;
        } else if (op.kind == hear_cnn::kPack) {
            const uint32_t n_p = (uint32_t)op.offs.size();
            const uint64_t ctw1 = 2ull * level * n;
            DevBuf prod((size_t)op.n_in * C * ctw * 8, st), y((size_t)op.n_in * C * ctw1 * 8, st),
                tmp((size_t)op.n_in * C * ctw1 * 8, st);
            mulplain(c, level, op.n_in * C, xin, op.mask.u64(), prod.u64(), st);
            rescale(c, level, 2 * op.n_in * C, prod.u64(), y.u64(), tmp.u64(), st);
            next = DevBuf((size_t)op.n_out * C * ctw1 * 8, st);
            std::vector<int32_t> back;
            for (uint32_t p = 1; p < n_p; p++) back.push_back(wrap(-(int64_t)op.offs[p], n / 2));
            DevBuf R((size_t)(n_p > 1 ? n_p - 1 : 1) * C * ctw1 * 8, st);
            for (uint32_t t = 0; t < op.n_out; t++) {
                const uint64_t *yt = y.u64() + (uint64_t)t * n_p * C * ctw1;
                uint64_t *ot = next.u64() + (uint64_t)t * C * ctw1;
                if (n_p == 1) {
                    HEAR_CHECK_CUDA(cudaMemcpyAsync(ot, yt, C * ctw1 * 8, cudaMemcpyDeviceToDevice, st));
                    continue;
                }
                rotate_each(c, level - 1, n_p - 1, C, yt + C * ctw1, rots_for(c, evk, back), R.u64(), st);
                sum_add_ct(c, level - 1, 2 * C, R.u64(), C * ctw1, n_p - 1, yt, ot, st);
            }
            const double ql = (double)c->primes[level];
            scale = scale * ql / ql;
        } else if (op.kind == hear_cnn::kRotsum) {
            const uint64_t words = (uint64_t)op.n_in * C * ctw;
            next = DevBuf(words * 8, st);
            HEAR_CHECK_CUDA(cudaMemcpyAsync(next.p, xin, words * 8, cudaMemcpyDeviceToDevice, st));
            DevBuf r(words * 8, st);
            for (int32_t s : op.steps) {
                rotate_each(c, level, 1, op.n_in * C, next.u64(), rots_for(c, evk, {s}), r.u64(), st);
                add_ct(c, level, 2 * op.n_in * C, next.u64(), r.u64(), next.u64(), st);
            }
        } else if (op.kind == hear_cnn::kQuad) {
            const uint32_t nc = op.n_in * C;
            const uint64_t ctw1 = 2ull * level * n, ctw2 = 2ull * (level - 1) * n;
            const uint64_t *bc = scaled_pts(m, k, scale, st);
            const uint64_t *Bp = bc, *Cp = bc + (size_t)op.n_in * level * n;
            // u = rescale(x (.) A) + B at level - 1
            DevBuf prod((size_t)nc * ctw * 8, st), u((size_t)nc * ctw1 * 8, st), tmp((size_t)nc * ctw1 * 8, st);
            mulplain_grouped(c, level, nc, C, xin, op.A.u64(), prod.u64(), st);
            rescale(c, level, 2 * nc, prod.u64(), u.u64(), tmp.u64(), st);
            add_plain(c, level - 1, nc, C, u.u64(), Bp, st);
            // x dropped to level - 1 (the last residue discarded, no division)
            DevBuf xd((size_t)nc * ctw1 * 8, st);
            HEAR_CHECK_CUDA(cudaMemcpy2DAsync(xd.p, (size_t)level * n * 8, xin, (size_t)L1 * n * 8,
                                              (size_t)level * n * 8, 2 * nc, cudaMemcpyDeviceToDevice, st));
            DevBuf v((size_t)nc * ctw1 * 8, st);
            mul_relin(c, level - 1, nc, xd.u64(), u.u64(), need_key(evk, 1), v.u64(), st);
            next = DevBuf((size_t)nc * ctw2 * 8, st);
            DevBuf tmp2((size_t)nc * ctw2 * 8, st);
            rescale(c, level - 1, 2 * nc, v.u64(), next.u64(), tmp2.u64(), st);
            add_plain(c, level - 2, nc, C, next.u64(), Cp, st);
            const double ql = (double)c->primes[level];
            const double su = scale * ql / ql;
            scale = scale * su / (double)c->primes[level - 1];
        } else {   // kBias
            const uint64_t words = (uint64_t)op.n_in * C * ctw;
            next = DevBuf(words * 8, st);
            HEAR_CHECK_CUDA(cudaMemcpyAsync(next.p, xin, words * 8, cudaMemcpyDeviceToDevice, st));
            add_plain(c, level, op.n_in * C, op.n_in * C, next.u64(), scaled_pts(m, k, scale, st), st);
        }
        cur = std::move(next);
        xin = cur.u64();
    }
    *scale_out = scale;
    return cur;
}

hear_cnn::Plan *cnn_graph_plan(const hear_cnn *m, const hear_eval_keys *evk, size_t op0, size_t op1, uint32_t C,
                               double scale_in, cudaStream_t st) {
    for (auto &p : m->plans)
        if (p->evk_serial == evk->serial && p->op0 == op0 && p->op1 == op1 && p->C == C && p->scale_in == scale_in)
            return p.get();
    hear_context *c = m->ctx;
    auto plan = std::make_unique<hear_cnn::Plan>();
    plan->evk_serial = evk->serial;
    plan->op0 = op0;
    plan->op1 = op1;
    plan->C = C;
    plan->scale_in = scale_in;
    const hear_cnn::Op &first = m->ops[op0], &last = m->ops[op1 - 1];
    const uint64_t in_words = (uint64_t)first.n_in * C * 2 * (first.level_in + 1) * c->n;
    const uint64_t out_words = (uint64_t)last.n_out * C * 2 * (last.level_out + 1) * c->n;
    plan->X = DevBuf(in_words * 8, nullptr);
    plan->Y = DevBuf(out_words * 8, nullptr);
    HEAR_CHECK_CUDA(cudaMemsetAsync(plan->X.p, 0, in_words * 8, st));
    {
        double so;
        DevBuf y = cnn_evaluate(m, evk, op0, op1, plan->X.u64(), C, scale_in, &so, st);
    }
    HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    cudaStream_t cs;
    HEAR_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const uint64_t launches0 = g_launches.load();
    cudaGraph_t graph = nullptr;
    HEAR_CHECK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    try {
        double so;
        DevBuf y = cnn_evaluate(m, evk, op0, op1, plan->X.u64(), C, scale_in, &so, cs);
        plan->scale_out = so;
        HEAR_CHECK_CUDA(cudaMemcpyAsync(plan->Y.p, y.p, out_words * 8, cudaMemcpyDeviceToDevice, cs));
    } catch (...) {
        cudaStreamEndCapture(cs, &graph);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        throw;
    }
    HEAR_CHECK_CUDA(cudaStreamEndCapture(cs, &graph));
    plan->launches = g_launches.load() - launches0;
    cudaError_t e = cudaGraphInstantiate(&plan->exec, graph, 0);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    HEAR_CHECK_CUDA(e);
    HEAR_CHECK_CUDA(cudaEventCreateWithFlags(&plan->done, cudaEventDisableTiming));
    m->plans.push_back(std::move(plan));
    return m->plans.back().get();
}

std::vector<double> cnn_pack_input(const hear_cnn *m, const double *x) {
    const uint32_t S = m->ctx->n / 2, dist = m->in_dist, cbar = S / dist;
    const uint32_t n_ct = m->in_kind == 1 ? 1 : m->in_c / cbar;
    const size_t plane = (size_t)m->in_h * m->in_w;
    std::vector<double> z((size_t)n_ct * S, 0.0);
    for (uint32_t i = 0; i < n_ct; i++)
        for (uint32_t mb = 0; mb < cbar; mb++) {
            const uint32_t ch = m->in_kind == 1 ? mb % m->in_c : cbar * i + mb;
            for (uint32_t y = 0; y < m->in_h; y++)
                for (uint32_t xx = 0; xx < m->in_w; xx++)
                    z[(size_t)i * S + (size_t)mb * dist + (size_t)y * m->in_pitch + xx] =
                        x[(size_t)ch * plane + (size_t)y * m->in_w + xx];
        }
    return z;
}

}  // namespace hear

hear_cnn::Plan::~Plan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (done) cudaEventDestroy(done);
}

namespace hear {
void set_last_error(const std::string &msg);   // capi.cu
}

// Host-only: the collapsed network's doubles (see collapse_layers), no context or GPU.
extern "C" hear_status hear_cnn_collapse(const hear_cnn_input *in, const hear_cnn_layer *layers, size_t n_layers,
                                         double *out, size_t cap, size_t *n) {
    using namespace hear;
    try {
        HEAR_REQUIRE(in && layers && n_layers, HEAR_E_INVAL, "no layers");
        HEAR_REQUIRE(in->conv_dims == 1 || in->conv_dims == 2, HEAR_E_INVAL, "conv_dims must be 1 or 2");
        const Collapsed col = collapse_layers(in, layers, n_layers);
        std::vector<double> v;
        uint32_t channels = in->c_in;
        for (const hear_cnn_layer &d : col.layers) {
            if (d.kind == HEAR_CNN_CONV) {
                v.insert(v.end(), d.w, d.w + (size_t)d.c_out * channels * d.f_h * d.f_w);
                channels = d.c_out;
            } else if (d.kind == HEAR_CNN_QUAD) {
                HEAR_REQUIRE(d.a && d.b && d.c, HEAR_E_INVAL, "quad needs a, b, c");
                for (const double *p : {d.a, d.b, d.c}) v.insert(v.end(), p, p + channels);
            } else if (d.kind == HEAR_CNN_FC) {
                v.insert(v.end(), d.w, d.w + (size_t)d.c_out * channels);
            }
        }
        if (n) *n = v.size();
        HEAR_REQUIRE(out && cap >= v.size(), HEAR_E_INVAL, "output capacity too small");
        std::copy(v.begin(), v.end(), out);
        return HEAR_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return HEAR_E_INVAL;
    }
}
