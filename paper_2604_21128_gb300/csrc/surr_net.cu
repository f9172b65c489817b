// The learned surrogate: a five-level convolutional operator that maps the
// E_z state and the medium of a lattice to the state K steps later, trained
// on trajectories the library computes, and the routine that uses it with
// plain QLA as fallback and arbiter (declared in qla.h, surr_*).
//
// Network (widths 32, 64, 128, 256, 256; 3x3 periodic convolutions, leaky
// ReLU 0.1, 2x2 average pooling down, nearest 2x upsampling up, additive
// skips):
//   E0 = a(conv(X))            E1 = a(conv(pool E0))  ...  E4 = a(conv(pool E3))
//   D3 = a(conv(up E4) + E3)   D2 = a(conv(up D3) + E2)  ...  D0 = a(conv(up D1) + E0)
//   Y  = conv(D0)              (3 outputs: the change of q2, q3, q4)
// Inputs: q2, q3, q4, n - 1.5, 4 dn/dx, 4 dn/dy (centred differences).
// BF16 weights and activations, FP32 accumulation, FP32 master weights,
// gradients and Adam state.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "qla_internal.h"
#include "surr_internal.h"

using namespace surr;

namespace {

constexpr int LEVELS = 5;
constexpr int WIDTH[LEVELS] = {32, 64, 128, 256, 256};
constexpr int FEAT = 6, NOUT = 3, CPAD = 32;
constexpr int NCONV = 10;

struct ConvSpec {
    int cin, cout, level;   // padded channel counts; level of its output
    int cin_real, cout_real;
    bool act, skip;
};

ConvSpec spec(int i) {
    // 0..4 encoder, 5..8 decoder (levels 3..0), 9 output
    if (i == 0) return {CPAD, WIDTH[0], 0, FEAT, WIDTH[0], true, false};
    if (i < 5) return {WIDTH[i - 1], WIDTH[i], i, WIDTH[i - 1], WIDTH[i], true, false};
    if (i < 9) {
        const int l = 8 - i;  // 3, 2, 1, 0
        return {WIDTH[l + 1], WIDTH[l], l, WIDTH[l + 1], WIDTH[l], true, true};
    }
    return {WIDTH[0], CPAD, 0, WIDTH[0], NOUT, false, false};
}

template <typename T>
T *carve(char *&p, size_t n) {
    T *r = reinterpret_cast<T *>(p);
    p += (n * sizeof(T) + 255) & ~size_t(255);
    return r;
}

}  // namespace

struct surr_net {
    int H = 0, W = 0, maxB = 0;
    cudaStream_t stream = nullptr;
    char *mem = nullptr;
    // parameters
    float *wf[NCONV], *bias[NCONV];           // master
    float *gw[NCONV], *gb[NCONV];             // gradients
    float *mw[NCONV], *vw[NCONV], *mb[NCONV], *vb[NCONV];
    bf16 *wb[NCONV], *wt[NCONV];              // bf16 copy, flipped-transposed copy
    size_t nw[NCONV];
    // activations (bf16), per level: E, D (l < 4), P (l >= 1), U (l < 4)
    bf16 *X, *E[LEVELS], *D[LEVELS], *Pl[LEVELS], *U[LEVELS];
    float *Y;                                  // [P0][CPAD]
    // gradients (fp32)
    float *dY, *dE[LEVELS], *dD[LEVELS], *dP[LEVELS], *dU[LEVELS];
    bf16 *dz;                                  // scratch
    float *part, *bpart;
    double *lpart;
    int lblocks = 0, bblocks = 0;
    long long step = 0;
    std::string err;
};

namespace {

qla_status nfail(surr_net *n, qla_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (n) n->err = buf;
    return s;
}

#define NCUDA(n, call, what)                                                        \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return nfail((n), QLA_ECUDA, "%s: %s", (what), cudaGetErrorString(e_)); \
    } while (0)

long long pixels(const surr_net *n, int B, int level) {
    return (long long)B * (n->H >> level) * (n->W >> level);
}

// Pixel splits of the weight gradient: one per 4096 pixels, at most 128
// (at 256^2 x 8 a cap of 32 left the level-0 gradient with too few CTAs:
// 4.85 ms per training step, 4.54 ms with 128).
int splits_for(long long P) {
    long long s = P / 4096;
    return int(std::max<long long>(1, std::min<long long>(128, s)));
}

size_t net_bytes(int H, int W, int B, bool with_mem, char **out_mem) {
    // Two passes: measure with a null base, then carve for real.
    (void)with_mem;
    (void)out_mem;
    size_t total = 0;
    auto add = [&](size_t bytes) { total += (bytes + 255) & ~size_t(255); };
    for (int i = 0; i < NCONV; ++i) {
        const ConvSpec s = spec(i);
        const size_t nw = size_t(s.cout) * 9 * s.cin;
        add(nw * 4 * 4);        // master, grad, m, v
        add(size_t(s.cout) * 4 * 4);
        add(nw * 2 * 2);        // bf16 copy + flipped copy
    }
    const long long P0 = (long long)B * H * W;
    add(P0 * CPAD * 2);                                    // X
    for (int l = 0; l < LEVELS; ++l) {
        const long long Pl = P0 >> (2 * l);
        add(Pl * WIDTH[l] * 2);                            // E
        if (l < 4) add(Pl * WIDTH[l] * 2);                 // D
        if (l >= 1) add(Pl * WIDTH[l - 1] * 2);            // P (input of E_l)
        if (l < 4) add(Pl * WIDTH[l + 1] * 2);             // U (input of D_l)
        add(Pl * WIDTH[l] * 4);                            // dE
        if (l < 4) add(Pl * WIDTH[l] * 4);                 // dD
        if (l >= 1) add(Pl * WIDTH[l - 1] * 4);            // dP
        if (l < 4) add(Pl * WIDTH[l + 1] * 4);             // dU
    }
    add(P0 * CPAD * 4 * 2);                                // Y, dY
    add(P0 * 256 * 2);                                     // dz scratch (>= any P_l * C_l)
    size_t part = 0;
    for (int i = 0; i < NCONV; ++i) {
        const ConvSpec s = spec(i);
        const long long Pin = P0 >> (2 * s.level);
        part = std::max(part, size_t(splits_for(Pin)) * s.cout * 9 * s.cin);
    }
    add(part * 4);
    add(1024 * 256 * 4);                                   // bias partials
    add(4096 * 8);                                         // loss partials
    return total;
}

void carve_all(surr_net *n, int B) {
    char *p = n->mem;
    for (int i = 0; i < NCONV; ++i) {
        const ConvSpec s = spec(i);
        const size_t nw = size_t(s.cout) * 9 * s.cin;
        n->nw[i] = nw;
        n->wf[i] = carve<float>(p, nw);
        n->gw[i] = carve<float>(p, nw);
        n->mw[i] = carve<float>(p, nw);
        n->vw[i] = carve<float>(p, nw);
        n->bias[i] = carve<float>(p, s.cout);
        n->gb[i] = carve<float>(p, s.cout);
        n->mb[i] = carve<float>(p, s.cout);
        n->vb[i] = carve<float>(p, s.cout);
        n->wb[i] = carve<bf16>(p, nw);
        n->wt[i] = carve<bf16>(p, nw);
    }
    const long long P0 = (long long)B * n->H * n->W;
    n->X = carve<bf16>(p, P0 * CPAD);
    for (int l = 0; l < LEVELS; ++l) {
        const long long Pl = P0 >> (2 * l);
        n->E[l] = carve<bf16>(p, Pl * WIDTH[l]);
        n->D[l] = l < 4 ? carve<bf16>(p, Pl * WIDTH[l]) : nullptr;
        n->Pl[l] = l >= 1 ? carve<bf16>(p, Pl * WIDTH[l - 1]) : nullptr;
        n->U[l] = l < 4 ? carve<bf16>(p, Pl * WIDTH[l + 1]) : nullptr;
        n->dE[l] = carve<float>(p, Pl * WIDTH[l]);
        n->dD[l] = l < 4 ? carve<float>(p, Pl * WIDTH[l]) : nullptr;
        n->dP[l] = l >= 1 ? carve<float>(p, Pl * WIDTH[l - 1]) : nullptr;
        n->dU[l] = l < 4 ? carve<float>(p, Pl * WIDTH[l + 1]) : nullptr;
    }
    n->Y = carve<float>(p, P0 * CPAD);
    n->dY = carve<float>(p, P0 * CPAD);
    n->dz = carve<bf16>(p, P0 * 256);
    size_t part = 0;
    for (int i = 0; i < NCONV; ++i) {
        const ConvSpec s = spec(i);
        const long long Pin = P0 >> (2 * s.level);
        part = std::max(part, size_t(splits_for(Pin)) * s.cout * 9 * s.cin);
    }
    n->part = carve<float>(p, part);
    n->bpart = carve<float>(p, 1024 * 256);
    n->lpart = carve<double>(p, 4096);
}

// conv layer i: its input tensor for batch B
const bf16 *conv_input(const surr_net *n, int i) {
    if (i == 0) return n->X;
    if (i < 5) return n->Pl[i];
    if (i < 9) return n->U[8 - i];
    return n->D[0];
}

bf16 *conv_output(surr_net *n, int i) {
    if (i < 5) return n->E[i];
    if (i < 9) return n->D[8 - i];
    return nullptr;
}

qla_status forward(surr_net *n, int B) {
    cudaStream_t st = n->stream;
    for (int i = 0; i < NCONV; ++i) {
        const ConvSpec s = spec(i);
        const int l = s.level;
        const int h = n->H >> l, w = n->W >> l;
        // inputs: pool before encoder levels >= 1, upsample before decoder
        if (i >= 1 && i < 5) {
            const long long m = pixels(n, B, l) * WIDTH[l - 1];
            k_pool<<<ew_blocks(m / 8), 256, 0, st>>>(n->E[l - 1], B, h * 2, w * 2, WIDTH[l - 1],
                                                 n->Pl[l]);
        } else if (i >= 5 && i < 9) {
            const bf16 *src = (i == 5) ? n->E[4] : n->D[l + 1];
            const long long m = pixels(n, B, l) * WIDTH[l + 1];
            k_up<<<ew_blocks(m / 8), 256, 0, st>>>(src, B, h / 2, w / 2, WIDTH[l + 1], n->U[l]);
        }
        NCUDA(n, cudaGetLastError(), "surrogate: resample");
        ConvArgs a{conv_input(n, i), B, h, w, s.cin, n->wb[i], s.cout, n->bias[i],
                   s.skip ? n->E[l] : nullptr, conv_output(n, i), n->Y};
        NCUDA(n, conv3x3(a, i == 9 ? OUT_F32 : OUT_BF16, s.act, s.skip, st), "surrogate: conv");
    }
    return QLA_OK;
}

// Backward through conv layer i given dOut (fp32) of its output.  Writes
// the weight and bias gradients, adds the pre-activation gradient to the
// skip tensor's gradient, and returns the input gradient in dIn (fp32,
// overwritten).
qla_status conv_backward(surr_net *n, int i, int B, const float *dOut, float *dSkip, float *dIn) {
    cudaStream_t st = n->stream;
    const ConvSpec s = spec(i);
    const int l = s.level, h = n->H >> l, w = n->W >> l;
    const long long P = pixels(n, B, l);
    const int blocks = int(std::min<long long>(1024, std::max<long long>(1, P / 256)));
    NCUDA(n, act_back(dOut, conv_output(n, i), P, s.cout, s.act, n->dz, dSkip, n->bpart, blocks, st),
          "surrogate: activation backward");
    NCUDA(n, sum_splits(n->bpart, blocks, s.cout, n->gb[i], st), "surrogate: bias grad");
    const int splits = splits_for(P);
    NCUDA(n, weight_grad(n->dz, conv_input(n, i), B, h, w, s.cout, s.cin, splits, n->part, st),
          "surrogate: weight grad");
    NCUDA(n, sum_splits(n->part, splits, (long long)s.cout * 9 * s.cin, n->gw[i], st),
          "surrogate: weight grad sum");
    if (dIn) {
        NCUDA(n, cudaMemsetAsync(dIn, 0, sizeof(float) * P * s.cin, st), "surrogate: clear");
        ConvArgs a{n->dz, B, h, w, s.cout, n->wt[i], s.cin, nullptr, nullptr, nullptr, dIn};
        NCUDA(n, conv3x3(a, ACC_F32, false, false, st), "surrogate: input grad");
    }
    return QLA_OK;
}

qla_status backward(surr_net *n, int B) {
    cudaStream_t st = n->stream;
    for (int i = 0; i < NCONV; ++i) {
        const ConvSpec s = spec(i);
        k_flip<<<ew_blocks(n->nw[i]), 256, 0, st>>>(n->wb[i], s.cout, s.cin, n->wt[i]);
    }
    NCUDA(n, cudaGetLastError(), "surrogate: flip");
    for (int l = 0; l < LEVELS; ++l) {
        NCUDA(n, cudaMemsetAsync(n->dE[l], 0, sizeof(float) * pixels(n, B, l) * WIDTH[l], st),
              "surrogate: clear");
    }
    qla_status r;
    // output conv: dY -> dD0
    if ((r = conv_backward(n, 9, B, n->dY, nullptr, n->dD[0])) != QLA_OK) return r;
    // decoder levels 0..3 (conv i = 8 - l): dD_l -> dU_l, skip into dE_l
    for (int l = 0; l < 4; ++l) {
        const int i = 8 - l;
        if ((r = conv_backward(n, i, B, n->dD[l], n->dE[l], n->dU[l])) != QLA_OK) return r;
        // up_l came from D_{l+1} (l < 3) or E4 (l = 3)
        const int h = n->H >> (l + 1), w = n->W >> (l + 1);
        float *dst = l < 3 ? n->dD[l + 1] : n->dE[4];
        const long long m = pixels(n, B, l + 1) * WIDTH[l + 1];
        if (l < 3) {
            k_up_back<<<ew_blocks(m / 4), 256, 0, st>>>(n->dU[l], B, h, w, WIDTH[l + 1], dst);
        } else {
            // dE4 only receives this gradient; D3's up-sampled input is E4
            k_up_back<<<ew_blocks(m / 4), 256, 0, st>>>(n->dU[l], B, h, w, WIDTH[l + 1], dst);
        }
        NCUDA(n, cudaGetLastError(), "surrogate: upsample backward");
    }
    // encoder levels 4..0: dE_l -> dP_l -> dE_{l-1} (accumulated)
    for (int l = 4; l >= 0; --l) {
        float *din = l >= 1 ? n->dP[l] : nullptr;
        if ((r = conv_backward(n, l, B, n->dE[l], nullptr, din)) != QLA_OK) return r;
        if (l >= 1) {
            const int H = n->H >> (l - 1), W = n->W >> (l - 1);
            const long long m = pixels(n, B, l - 1) * WIDTH[l - 1];
            k_pool_back<<<ew_blocks(m / 4), 256, 0, st>>>(n->dP[l], B, H, W, WIDTH[l - 1], n->dE[l - 1]);
            NCUDA(n, cudaGetLastError(), "surrogate: pool backward");
        }
    }
    return QLA_OK;
}

// After a stream synchronisation: did a tcgen05 convolution give up one of
// its bounded waits since the last check?  (Its CTAs then skipped their
// epilogues, so the outputs are not to be trusted.)
qla_status tc_waits_ok(surr_net *n) {
    int flag = 0;
    NCUDA(n, conv_tc_error(&flag, true), "surrogate: wait flag");
    if (flag)
        return nfail(n, QLA_ETIMEOUT,
                     "surrogate: a tensor-core wait ran out; results of tensor-core launches "
                     "are undefined until the network is rebuilt");
    return QLA_OK;
}

qla_status loss(surr_net *n, int B, const float *target, double *out) {
    const long long P = pixels(n, B, 0);
    const int blocks = std::min(n->lblocks, ew_blocks(P));
    k_mse<<<blocks, 256, 0, n->stream>>>(n->Y, CPAD, target, NOUT, P, n->dY, n->lpart);
    NCUDA(n, cudaGetLastError(), "surrogate: loss");
    std::vector<double> h(blocks);
    NCUDA(n, cudaMemcpyAsync(h.data(), n->lpart, sizeof(double) * blocks, cudaMemcpyDeviceToHost,
                             n->stream), "surrogate: loss copy");
    NCUDA(n, cudaStreamSynchronize(n->stream), "surrogate: sync");
    const qla_status w = tc_waits_ok(n);
    if (w != QLA_OK) return w;
    double s = 0.0;
    for (double v : h) s += v;
    *out = s;
    return QLA_OK;
}

qla_status pack(surr_net *n, const float *feat, int B) {
    const long long P = pixels(n, B, 0);
    k_pack_in<<<ew_blocks(P), 256, 0, n->stream>>>(feat, P, FEAT, CPAD, n->X);
    NCUDA(n, cudaGetLastError(), "surrogate: pack");
    return QLA_OK;
}

qla_status check_batch(surr_net *n, int B) {
    if (B < 1 || B > n->maxB) return nfail(n, QLA_EINVAL, "batch %d outside 1..%d", B, n->maxB);
    return QLA_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Lattice side: features, candidate checks, the window loop with fallback.
// ---------------------------------------------------------------------------
namespace {

// Features of an FP32 E_z context (the state with the pending potential
// step applied, and the medium): [ny][nx][6].
__global__ void k_features(const float *__restrict__ q, size_t plane, int nx, int ny, int pitch,
                           bool vin, const uint32_t *__restrict__ midx,
                           const qla::MedRec<float> *__restrict__ table,
                           const double *__restrict__ n, float *__restrict__ f) {
    const size_t N = size_t(nx) * ny;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        const size_t g = size_t(j) * pitch + i;
        float s[6];
        qla::load_site<float, 3, qla::V_ROTATION>(q, plane, g, vin, midx, table, s);
        const double dnx = 0.5 * (n[size_t(j) * pitch + qla::wrap(i + 1, nx)] -
                                  n[size_t(j) * pitch + qla::wrap(i - 1, nx)]);
        const double dny = 0.5 * (n[size_t(qla::wrap(j + 1, ny)) * pitch + i] -
                                  n[size_t(qla::wrap(j - 1, ny)) * pitch + i]);
        float *o = f + t * FEAT;
        o[0] = s[2];
        o[1] = s[3];
        o[2] = s[4];
        o[3] = float(n[g] - 1.5);
        o[4] = float(4.0 * dnx);
        o[5] = float(4.0 * dny);
    }
}

// candidate q = q(t) (from the features) + y; energy and the change of the
// discrete divergence of B (centred differences) against q(t)'s, as sums.
__global__ void k_candidate(const float *__restrict__ f, const float *__restrict__ y, int nx,
                            int ny, float *__restrict__ cand, double *__restrict__ sums) {
    __shared__ double red[3][256];
    const size_t N = size_t(nx) * ny;
    double e = 0.0, dd = 0.0, gg = 0.0;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        float c[3];
        for (int k = 0; k < 3; ++k) {
            c[k] = f[t * FEAT + k] + y[t * NOUT + k];
            cand[k * N + t] = c[k];
            e += double(c[k]) * c[k];
        }
        auto at = [&](int ii, int jj, int k) {
            const size_t s = size_t(qla::wrap(jj, ny)) * nx + qla::wrap(ii, nx);
            return double(f[s * FEAT + k]) + double(y[s * NOUT + k]);
        };
        auto at0 = [&](int ii, int jj, int k) {
            const size_t s = size_t(qla::wrap(jj, ny)) * nx + qla::wrap(ii, nx);
            return double(f[s * FEAT + k]);
        };
        // B_x = q3 (index 1), B_y = q4 (index 2)
        const double dbx = 0.5 * (at(i + 1, j, 1) - at(i - 1, j, 1));
        const double dby = 0.5 * (at(i, j + 1, 2) - at(i, j - 1, 2));
        const double d0 = 0.5 * (at0(i + 1, j, 1) - at0(i - 1, j, 1)) +
                          0.5 * (at0(i, j + 1, 2) - at0(i, j - 1, 2));
        const double dv = dbx + dby - d0;
        dd += dv * dv;
        gg += dbx * dbx + dby * dby;
    }
    red[0][threadIdx.x] = e;
    red[1][threadIdx.x] = dd;
    red[2][threadIdx.x] = gg;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) sums[blockIdx.x * 3 + k] = red[k][0];
}

// Write a candidate (three contiguous planes q2, q3, q4) as the state.
__global__ void k_store_candidate(const float *__restrict__ cand, int nx, int ny, int pitch,
                                  size_t plane, float *__restrict__ q) {
    const size_t N = size_t(nx) * ny;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        const size_t g = size_t(j) * pitch + i;
        for (int k = 0; k < 3; ++k) q[k * plane + g] = cand[k * N + t];
    }
}

qla_status ctx_ok(qla_ctx *c) {
    if (!c) return QLA_EINVAL;
    if (c->sticky != QLA_OK) return c->sticky;
    if (c->prec != QLA_FP32 || c->P != 3 || c->vmode != qla::V_ROTATION) return QLA_EINVAL;
    if (!c->has_medium || !c->has_state) return QLA_ESTATE;
    return QLA_OK;
}

}  // namespace

extern "C" {

size_t surr_workspace_bytes(int height, int width, int max_batch) {
    if (height < 16 || width < 16 || height % 16 || width % 16 || max_batch < 1) return 0;
    // the elementwise kernels index the widest level-0 tensor with 32 bits
    if ((long long)max_batch * height * width * 32 >= (1LL << 31)) return 0;
    return net_bytes(height, width, max_batch, false, nullptr);
}

qla_status surr_create(surr_net **out, int height, int width, int max_batch,
                       unsigned long long seed, void *cuda_stream, void *workspace,
                       size_t workspace_bytes) {
    if (!out) return QLA_EINVAL;
    *out = nullptr;
    const size_t need = surr_workspace_bytes(height, width, max_batch);
    if (need == 0) return QLA_EINVAL;
    if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return QLA_EINVAL;
    surr_net *n = new (std::nothrow) surr_net();
    if (!n) return QLA_ENOMEM;
    n->H = height;
    n->W = width;
    n->maxB = max_batch;
    n->stream = static_cast<cudaStream_t>(cuda_stream);
    n->mem = static_cast<char *>(workspace);
    carve_all(n, max_batch);
    n->lblocks = 4096;
    // He-style initialisation from a seeded generator (host), zero biases
    std::mt19937_64 rng(seed);
    for (int i = 0; i < NCONV; ++i) {
        const ConvSpec s = spec(i);
        std::vector<float> w(n->nw[i], 0.f);
        const double fan_in = 9.0 * s.cin_real;
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / fan_in) * (i == 9 ? 0.1 : 1.0));
        for (int co = 0; co < s.cout_real; ++co)
            for (int t = 0; t < 9; ++t)
                for (int ci = 0; ci < s.cin_real; ++ci)
                    w[(size_t(co) * 9 + t) * s.cin + ci] = float(nd(rng));
        std::vector<float> zeros(s.cout, 0.f);
        if (cudaMemcpyAsync(n->wf[i], w.data(), n->nw[i] * 4, cudaMemcpyHostToDevice, n->stream) ||
            cudaMemsetAsync(n->bias[i], 0, s.cout * 4, n->stream) ||
            cudaMemsetAsync(n->mw[i], 0, n->nw[i] * 4, n->stream) ||
            cudaMemsetAsync(n->vw[i], 0, n->nw[i] * 4, n->stream) ||
            cudaMemsetAsync(n->mb[i], 0, s.cout * 4, n->stream) ||
            cudaMemsetAsync(n->vb[i], 0, s.cout * 4, n->stream) ||
            cudaStreamSynchronize(n->stream)) {
            delete n;
            return QLA_ECUDA;
        }
        k_to_bf16<<<ew_blocks(n->nw[i]), 256, 0, n->stream>>>(n->wf[i], n->nw[i], n->wb[i]);
    }
    if (cudaStreamSynchronize(n->stream) != cudaSuccess) {
        delete n;
        return QLA_ECUDA;
    }
    *out = n;
    return QLA_OK;
}

long long surr_param_count(const surr_net *n) {
    (void)n;
    long long c = 0;
    for (int i = 0; i < NCONV; ++i) {
        const ConvSpec s = spec(i);
        c += (long long)s.cout_real * s.cin_real * 9 + s.cout_real;
    }
    return c;
}

// Host layout, per conv layer: weights (cout, cin, 3, 3) then bias (cout),
// real channel counts; ky, kx = dy + 1, dx + 1.
static qla_status params_io(surr_net *n, float *host, bool get, bool grads) {
    if (!n || !host) return QLA_EINVAL;
    size_t off = 0;
    for (int i = 0; i < NCONV; ++i) {
        const ConvSpec s = spec(i);
        std::vector<float> w(n->nw[i]), b(s.cout);
        float *dw = grads ? n->gw[i] : n->wf[i];
        float *db = grads ? n->gb[i] : n->bias[i];
        if (get || true) {
            NCUDA(n, cudaMemcpyAsync(w.data(), dw, n->nw[i] * 4, cudaMemcpyDeviceToHost, n->stream),
                  "surrogate: params");
            NCUDA(n, cudaMemcpyAsync(b.data(), db, s.cout * 4, cudaMemcpyDeviceToHost, n->stream),
                  "surrogate: params");
            NCUDA(n, cudaStreamSynchronize(n->stream), "surrogate: sync");
        }
        for (int co = 0; co < s.cout_real; ++co)
            for (int ci = 0; ci < s.cin_real; ++ci)
                for (int t = 0; t < 9; ++t) {
                    float &d = w[(size_t(co) * 9 + t) * s.cin + ci];
                    float &h = host[off + (size_t(co) * s.cin_real + ci) * 9 + t];
                    if (get) h = d; else d = h;
                }
        off += size_t(s.cout_real) * s.cin_real * 9;
        for (int co = 0; co < s.cout_real; ++co) {
            if (get) host[off + co] = b[co]; else b[co] = host[off + co];
        }
        off += s.cout_real;
        if (!get) {
            NCUDA(n, cudaMemcpyAsync(dw, w.data(), n->nw[i] * 4, cudaMemcpyHostToDevice, n->stream),
                  "surrogate: params");
            NCUDA(n, cudaMemcpyAsync(db, b.data(), s.cout * 4, cudaMemcpyHostToDevice, n->stream),
                  "surrogate: params");
            k_to_bf16<<<ew_blocks(n->nw[i]), 256, 0, n->stream>>>(n->wf[i], n->nw[i], n->wb[i]);
            NCUDA(n, cudaStreamSynchronize(n->stream), "surrogate: sync");
        }
    }
    return QLA_OK;
}

qla_status surr_get_params(surr_net *n, float *host) { return params_io(n, host, true, false); }
qla_status surr_set_params(surr_net *n, const float *host) {
    return params_io(n, const_cast<float *>(host), false, false);
}

qla_status surr_forward(surr_net *n, const float *feat_dev, int B, float *out_dev) {
    if (!n || !feat_dev || !out_dev) return QLA_EINVAL;
    qla_status s = check_batch(n, B);
    if (s != QLA_OK) return s;
    if ((s = pack(n, feat_dev, B)) != QLA_OK) return s;
    if ((s = forward(n, B)) != QLA_OK) return s;
    const long long P = pixels(n, B, 0);
    k_strip<<<ew_blocks(P * NOUT), 256, 0, n->stream>>>(n->Y, CPAD, NOUT, P, out_dev);
    NCUDA(n, cudaGetLastError(), "surrogate: strip");
    return QLA_OK;
}

qla_status surr_loss_grad(surr_net *n, const float *feat_dev, const float *target_dev, int B,
                          double *loss_out, float *grad_host) {
    if (!n || !feat_dev || !target_dev) return QLA_EINVAL;
    qla_status s = check_batch(n, B);
    if (s != QLA_OK) return s;
    if ((s = pack(n, feat_dev, B)) != QLA_OK) return s;
    if ((s = forward(n, B)) != QLA_OK) return s;
    double l = 0.0;
    if ((s = loss(n, B, target_dev, &l)) != QLA_OK) return s;
    if (loss_out) *loss_out = l;
    if ((s = backward(n, B)) != QLA_OK) return s;
    if (grad_host) return params_io(n, grad_host, true, true);
    return QLA_OK;
}

qla_status surr_train_step(surr_net *n, const float *feat_dev, const float *target_dev, int B,
                           float lr, double *loss_out) {
    qla_status s = surr_loss_grad(n, feat_dev, target_dev, B, loss_out, nullptr);
    if (s != QLA_OK) return s;
    n->step++;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = float(1.0 - std::pow(0.9, double(n->step)));
    const float c2 = float(1.0 - std::pow(0.999, double(n->step)));
    for (int i = 0; i < NCONV; ++i) {
        const ConvSpec sp = spec(i);
        k_adam<<<ew_blocks(n->nw[i]), 256, 0, n->stream>>>(n->wf[i], n->gw[i], n->mw[i], n->vw[i],
                                                           n->nw[i], lr, b1, b2, eps, c1, c2,
                                                           n->wb[i]);
        k_adam<<<1, 256, 0, n->stream>>>(n->bias[i], n->gb[i], n->mb[i], n->vb[i], sp.cout, lr, b1,
                                         b2, eps, c1, c2, nullptr);
    }
    NCUDA(n, cudaGetLastError(), "surrogate: adam");
    return QLA_OK;
}

const char *surr_last_error(const surr_net *n) { return n ? n->err.c_str() : "null network"; }

void surr_destroy(surr_net *n) {
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    delete n;
}

qla_status surr_features(qla_ctx *c, float *feat_dev) {
    qla_status s = ctx_ok(c);
    if (s != QLA_OK) return s;
    if (!feat_dev) return QLA_EINVAL;
    const size_t N = size_t(c->nx) * c->ny;
    k_features<<<int(std::min<size_t>((N + 255) / 256, 8192)), 256, 0, c->stream>>>(
        static_cast<const float *>(c->state[c->cur]), c->plane_elems, c->nx, c->ny, c->pitch,
        c->pending_v, c->midx, static_cast<const qla::MedRec<float> *>(c->table), c->n, feat_dev);
    return cudaGetLastError() == cudaSuccess ? QLA_OK : QLA_ECUDA;
}

qla_status surr_advance(qla_ctx *c, surr_net *n, int windows, int K, double energy_tol,
                        double div_tol, float *scratch_dev, int *accepted, double *energies) {
    qla_status s = ctx_ok(c);
    if (s != QLA_OK) return s;
    if (!n || !scratch_dev || windows < 0 || K < 1 || n->H != c->ny || n->W != c->nx)
        return QLA_EINVAL;
    const size_t N = size_t(c->nx) * c->ny;
    float *feat = scratch_dev, *y = feat + N * FEAT, *cand = y + N * NOUT;
    const int blocks = 256;
    double *sums = n->lpart;  // blocks * 3 doubles
    int acc = 0;
    for (int wdx = 0; wdx < windows; ++wdx) {
        double e0 = 0.0;
        if ((s = qla_energy(c, &e0)) != QLA_OK) return s;
        if ((s = surr_features(c, feat)) != QLA_OK) return s;
        if ((s = surr_forward(n, feat, 1, y)) != QLA_OK) return s;
        k_candidate<<<blocks, 256, 0, c->stream>>>(feat, y, c->nx, c->ny, cand, sums);
        std::vector<double> h(size_t(blocks) * 3);
        if (cudaMemcpyAsync(h.data(), sums, h.size() * 8, cudaMemcpyDeviceToHost, c->stream) ||
            cudaStreamSynchronize(c->stream))
            return QLA_ECUDA;
        if ((s = tc_waits_ok(n)) != QLA_OK) return s;
        double e1 = 0.0, dd = 0.0, gg = 0.0;
        for (int b = 0; b < blocks; ++b) {
            e1 += h[b * 3];
            dd += h[b * 3 + 1];
            gg += h[b * 3 + 2];
        }
        const bool ok = std::fabs(e1 / e0 - 1.0) <= energy_tol &&
                        std::sqrt(dd / (gg > 0 ? gg : 1e-300)) <= div_tol;
        if (ok) {
            k_store_candidate<<<int(std::min<size_t>((N + 255) / 256, 8192)), 256, 0, c->stream>>>(
                cand, c->nx, c->ny, c->pitch, c->plane_elems, static_cast<float *>(c->state[c->cur]));
            if (cudaGetLastError() != cudaSuccess) return QLA_ECUDA;
            c->pending_v = false;
            ++acc;
        } else {
            if ((s = qla_step(c, K)) != QLA_OK) return s;
        }
        if (energies && (s = qla_energy(c, energies + wdx)) != QLA_OK) return s;
    }
    if (accepted) *accepted = acc;
    return QLA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Direct access to the two contraction kernels, for exactness tests: with
// BF16 inputs their only rounding is the FP32 accumulation.
// ---------------------------------------------------------------------------
extern "C" qla_status surr_conv3x3_raw(const void *in_bf16, int B, int H, int W, int cin,
                                       const void *w_bf16, int cout, float *out_f32,
                                       void *cuda_stream) {
    if (!in_bf16 || !w_bf16 || !out_f32 || B < 1 || H < 1 || W < 1 || cin % 32 || cout % 32)
        return QLA_EINVAL;
    ConvArgs a{static_cast<const bf16 *>(in_bf16), B, H, W, cin, static_cast<const bf16 *>(w_bf16),
               cout, nullptr, nullptr, nullptr, out_f32};
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (conv3x3(a, OUT_F32, false, false, st) != cudaSuccess) return QLA_ECUDA;
    int flag = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess || conv_tc_error(&flag, true) != cudaSuccess)
        return QLA_ECUDA;
    return flag ? QLA_ETIMEOUT : QLA_OK;
}

extern "C" qla_status surr_test_stall_conv(int on) {
    return conv_tc_stall(on ? 1 : 0) == cudaSuccess ? QLA_OK : QLA_ECUDA;
}

extern "C" qla_status surr_weight_grad_raw(const void *dz_bf16, const void *in_bf16, int B, int H,
                                           int W, int cout, int cin, int splits, float *part,
                                           float *dw_f32, void *cuda_stream) {
    if (!dz_bf16 || !in_bf16 || !part || !dw_f32 || cin % 32 || cout % 32 || splits < 1)
        return QLA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (weight_grad(static_cast<const bf16 *>(dz_bf16), static_cast<const bf16 *>(in_bf16), B, H, W,
                    cout, cin, splits, part, st) != cudaSuccess)
        return QLA_ECUDA;
    return sum_splits(part, splits, (long long)cout * 9 * cin, dw_f32, st) == cudaSuccess
               ? QLA_OK : QLA_ECUDA;
}
