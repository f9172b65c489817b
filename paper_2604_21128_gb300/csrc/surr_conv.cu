// Convolution kernels of the learned surrogate: 3x3 periodic convolution as
// an implicit GEMM on the tensor cores (forward, and input gradient with
// flipped, transposed weights), weight gradient as a split-K GEMM over the
// pixels with a fixed-order reduction, and the elementwise kernels around
// them.  All tensors are NHWC; channel counts are multiples of 32.
#include "surr_internal.h"

namespace surr {

// ---------------------------------------------------------------------------
// Forward / input-gradient convolution.
//   out[p, co] = sum_{tap, ci} w[co][tap][ci] * in[p shifted by tap, ci]
// p = (b, y, x) flattened; tap = 3 (dy + 1) + (dx + 1); periodic in y, x.
// CTA tile 64 pixels x NT output channels, 4 warps (2 x 2), K in steps of 16
// channels of one tap, double-buffered with cp.async.  Epilogue by MODE:
//   OUT_BF16: out_bf = act(acc + bias + skip)   (act optional)
//   OUT_F32 : out_f  = acc + bias
//   ACC_F32 : out_f += acc
// ---------------------------------------------------------------------------
constexpr int CTM = 64;     // pixels per CTA
constexpr int KS = 16;      // channels per K step
constexpr int APAD = 24;    // smem row stride (elements): 48 bytes, ldmatrix conflict-free

template <int NT, int MODE, bool ACT, bool SKIP>
__global__ void __launch_bounds__(128)
k_conv3x3(const bf16 *__restrict__ in, int B, int H, int W, int cin,
          const bf16 *__restrict__ w, int cout, const float *__restrict__ bias,
          const bf16 *__restrict__ skip, bf16 *__restrict__ out_bf, float *__restrict__ out_f) {
    __shared__ __align__(16) bf16 As[2][CTM][APAD];
    __shared__ __align__(16) bf16 Bs[2][NT][APAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const long long P = (long long)B * H * W;
    const long long p0 = (long long)blockIdx.x * CTM;
    const int co0 = blockIdx.y * NT;

    // this thread's A row (pixel) and half (8 channels)
    const int ar = tid >> 1, ah = tid & 1;
    const long long pa = p0 + ar;
    int ab = 0, ay = 0, ax = 0;
    const bool a_ok = pa < P;
    if (a_ok) {
        ab = int(pa / (H * W));
        const int rem = int(pa - (long long)ab * H * W);
        ay = rem / W;
        ax = rem - ay * W;
    }
    const int kchunks = cin / KS;
    const int ksteps = 9 * kchunks;

    auto load = [&](int s, int kstep) {
        const int tap = kstep / kchunks, ci0 = (kstep - tap * kchunks) * KS;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        if (a_ok) {
            const long long ps = (long long)ab * H * W + (long long)wrapi(ay + dy, H) * W +
                                 wrapi(ax + dx, W);
            cp16(&As[s][ar][ah * 8], in + ps * cin + ci0 + ah * 8);
        } else {
            *reinterpret_cast<uint4 *>(&As[s][ar][ah * 8]) = make_uint4(0, 0, 0, 0);
        }
        for (int c = tid; c < NT * 2; c += 128) {
            const int n = c >> 1, h = c & 1;
            cp16(&Bs[s][n][h * 8], w + ((long long)(co0 + n) * 9 + tap) * cin + ci0 + h * 8);
        }
        cp_commit();
    };

    constexpr int NI = NT / 16;  // n8 tiles per warp (each warp covers NT / 2 channels)
    float acc[2][NI][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NI; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    load(0, 0);
    for (int ks = 0; ks < ksteps; ++ks) {
        const int s = ks & 1;
        if (ks + 1 < ksteps) {
            load(s ^ 1, ks + 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        unsigned a[2][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
            ldsm_x4(a[mi], &As[s][wm * 32 + mi * 16 + (lane & 15)][(lane >> 4) * 8]);
#pragma unroll
        for (int nj = 0; nj < NI / 2; ++nj) {
            unsigned bfr[4];
            ldsm_x4(bfr, &Bs[s][wn * (NT / 2) + nj * 16 + (lane & 7) + ((lane >> 4) << 3)]
                          [((lane >> 3) & 1) * 8]);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                mma_bf16(acc[mi][2 * nj], a[mi], bfr[0], bfr[1]);
                mma_bf16(acc[mi][2 * nj + 1], a[mi], bfr[2], bfr[3]);
            }
        }
        __syncthreads();
    }

    // epilogue
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const long long p = p0 + wm * 32 + mi * 16 + (lane >> 2) + half * 8;
            if (p >= P) continue;
#pragma unroll
            for (int ni = 0; ni < NI; ++ni) {
                const int co = co0 + wn * (NT / 2) + ni * 8 + (lane & 3) * 2;
                float v0 = acc[mi][ni][half * 2], v1 = acc[mi][ni][half * 2 + 1];
                if constexpr (MODE == OUT_BF16) {
                    if (bias) { v0 += bias[co]; v1 += bias[co + 1]; }
                    if constexpr (SKIP) {
                        const __nv_bfloat162 sk =
                            *reinterpret_cast<const __nv_bfloat162 *>(skip + p * cout + co);
                        v0 += __bfloat162float(sk.x);
                        v1 += __bfloat162float(sk.y);
                    }
                    if constexpr (ACT) {
                        v0 = v0 > 0.f ? v0 : LEAK * v0;
                        v1 = v1 > 0.f ? v1 : LEAK * v1;
                    }
                    *reinterpret_cast<__nv_bfloat162 *>(out_bf + p * cout + co) =
                        __floats2bfloat162_rn(v0, v1);
                } else if constexpr (MODE == OUT_F32) {
                    if (bias) { v0 += bias[co]; v1 += bias[co + 1]; }
                    *reinterpret_cast<float2 *>(out_f + p * cout + co) = make_float2(v0, v1);
                } else {
                    float2 *o = reinterpret_cast<float2 *>(out_f + p * cout + co);
                    const float2 prev = *o;
                    *o = make_float2(prev.x + v0, prev.y + v1);
                }
            }
        }
    }
}

template <int MODE, bool ACT, bool SKIP>
static cudaError_t conv_t(const ConvArgs &a, cudaStream_t st) {
    const long long P = (long long)a.B * a.H * a.W;
    const int nt = (a.cout % 64 == 0) ? 64 : 32;
    dim3 grid(unsigned((P + CTM - 1) / CTM), unsigned(a.cout / nt));
    if (nt == 64)
        k_conv3x3<64, MODE, ACT, SKIP><<<grid, 128, 0, st>>>(a.in, a.B, a.H, a.W, a.cin, a.w,
                                                            a.cout, a.bias, a.skip, a.out_bf,
                                                            a.out_f);
    else
        k_conv3x3<32, MODE, ACT, SKIP><<<grid, 128, 0, st>>>(a.in, a.B, a.H, a.W, a.cin, a.w,
                                                            a.cout, a.bias, a.skip, a.out_bf,
                                                            a.out_f);
    return cudaGetLastError();
}

cudaError_t conv3x3(const ConvArgs &a, int mode, bool act, bool skip, cudaStream_t st) {
    if (a.cin % 32 || a.cout % 32) return cudaErrorInvalidValue;
    if (mode == OUT_BF16) {
        if (act) return skip ? conv_t<OUT_BF16, true, true>(a, st) : conv_t<OUT_BF16, true, false>(a, st);
        return skip ? conv_t<OUT_BF16, false, true>(a, st) : conv_t<OUT_BF16, false, false>(a, st);
    }
    if (mode == OUT_F32) return conv_t<OUT_F32, false, false>(a, st);
    return conv_t<ACC_F32, false, false>(a, st);
}

// ---------------------------------------------------------------------------
// Weight gradient: part[split][co][tap][ci] = sum over this split's pixels p
// of dz[p][co] * in[p shifted by tap][ci].  CTA tile 64 co x 64 ci (or 32),
// 4 warps (2 x 2), 64 pixels per stage (4 K steps of 16), operands loaded
// pixel-major and fed to the MMA with transposing ldmatrix.
// ---------------------------------------------------------------------------
constexpr int DWK = 64;   // pixels per stage

template <int MT, int NT>
__global__ void __launch_bounds__(128)
k_dw(const bf16 *__restrict__ dz, const bf16 *__restrict__ in, int B, int H, int W, int cout,
     int cin, long long pix_per_split, float *__restrict__ part) {
    __shared__ __align__(16) bf16 As[2][DWK][MT + 8];
    __shared__ __align__(16) bf16 Bs[2][DWK][NT + 8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int ci0 = blockIdx.x * NT, co0 = blockIdx.y * MT;
    const int splits = int(gridDim.z / 9);
    const int tap = blockIdx.z / splits, split = blockIdx.z - tap * splits;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const long long P = (long long)B * H * W;
    const long long q0 = split * pix_per_split;
    long long q1 = q0 + pix_per_split;
    if (q1 > P) q1 = P;

    auto load = [&](int s, long long pb) {
        constexpr int ACH = MT / 8, BCH = NT / 8;
        for (int c = tid; c < DWK * ACH; c += 128) {
            const int r = c / ACH, h = c - r * ACH;
            const long long p = pb + r;
            if (p < q1) cp16(&As[s][r][h * 8], dz + p * cout + co0 + h * 8);
            else *reinterpret_cast<uint4 *>(&As[s][r][h * 8]) = make_uint4(0, 0, 0, 0);
        }
        for (int c = tid; c < DWK * BCH; c += 128) {
            const int r = c / BCH, h = c - r * BCH;
            const long long p = pb + r;
            if (p < q1) {
                const int b = int(p / (H * W));
                const int rem = int(p - (long long)b * H * W);
                const int y = rem / W, x = rem - y * W;
                const long long ps = (long long)b * H * W + (long long)wrapi(y + dy, H) * W +
                                     wrapi(x + dx, W);
                cp16(&Bs[s][r][h * 8], in + ps * cin + ci0 + h * 8);
            } else {
                *reinterpret_cast<uint4 *>(&Bs[s][r][h * 8]) = make_uint4(0, 0, 0, 0);
            }
        }
        cp_commit();
    };

    constexpr int MI = MT / 32, NI = NT / 16;  // per warp: MT/2 rows, NT/2 cols
    float acc[MI][NI][4];
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < NI; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    const long long nst = (q1 - q0 + DWK - 1) / DWK;
    if (nst > 0) load(0, q0);
    for (long long st = 0; st < nst; ++st) {
        const int s = int(st & 1);
        if (st + 1 < nst) {
            load(s ^ 1, q0 + (st + 1) * DWK);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < DWK / 16; ++kk) {
            unsigned a[MI][4];
#pragma unroll
            for (int mi = 0; mi < MI; ++mi)
                ldsm_x4_t(a[mi], &As[s][kk * 16 + (lane & 7) + ((lane >> 4) << 3)]
                                   [wm * (MT / 2) + mi * 16 + ((lane >> 3) & 1) * 8]);
#pragma unroll
            for (int nj = 0; nj < NI / 2; ++nj) {
                unsigned bfr[4];
                ldsm_x4_t(bfr, &Bs[s][kk * 16 + (lane & 7) + ((lane >> 3) & 1) * 8]
                                 [wn * (NT / 2) + nj * 16 + ((lane >> 4) << 3)]);
#pragma unroll
                for (int mi = 0; mi < MI; ++mi) {
                    mma_bf16(acc[mi][2 * nj], a[mi], bfr[0], bfr[1]);
                    mma_bf16(acc[mi][2 * nj + 1], a[mi], bfr[2], bfr[3]);
                }
            }
        }
        __syncthreads();
    }
    // part layout: [split][co][tap][ci]
#pragma unroll
    for (int mi = 0; mi < MI; ++mi)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int co = co0 + wm * (MT / 2) + mi * 16 + (lane >> 2) + half * 8;
#pragma unroll
            for (int ni = 0; ni < NI; ++ni) {
                const int ci = ci0 + wn * (NT / 2) + ni * 8 + (lane & 3) * 2;
                float *o = part + (((long long)split * cout + co) * 9 + tap) * cin + ci;
                *reinterpret_cast<float2 *>(o) =
                    make_float2(acc[mi][ni][half * 2], acc[mi][ni][half * 2 + 1]);
            }
        }
}

cudaError_t weight_grad(const bf16 *dz, const bf16 *in, int B, int H, int W, int cout, int cin,
                        int splits, float *part, cudaStream_t st) {
    if (cin % 32 || cout % 32 || splits < 1) return cudaErrorInvalidValue;
    const long long P = (long long)B * H * W;
    long long per = (P + splits - 1) / splits;
    per = (per + DWK - 1) / DWK * DWK;
    const int mt = cout % 64 == 0 ? 64 : 32, nt = cin % 64 == 0 ? 64 : 32;
    dim3 grid(unsigned(cin / nt), unsigned(cout / mt), unsigned(9 * splits));
    if (mt == 64 && nt == 64) k_dw<64, 64><<<grid, 128, 0, st>>>(dz, in, B, H, W, cout, cin, per, part);
    else if (mt == 64) k_dw<64, 32><<<grid, 128, 0, st>>>(dz, in, B, H, W, cout, cin, per, part);
    else if (nt == 64) k_dw<32, 64><<<grid, 128, 0, st>>>(dz, in, B, H, W, cout, cin, per, part);
    else k_dw<32, 32><<<grid, 128, 0, st>>>(dz, in, B, H, W, cout, cin, per, part);
    return cudaGetLastError();
}

// Sum the split partials in split order into g.
__global__ void k_sum_splits(const float *__restrict__ part, int splits, long long n,
                             float *__restrict__ g) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < splits; ++k) s += part[k * n + i];
        g[i] = s;
    }
}

cudaError_t sum_splits(const float *part, int splits, long long n, float *g, cudaStream_t st) {
    const int blocks = int(std::min<long long>((n + 255) / 256, 4096));
    k_sum_splits<<<blocks, 256, 0, st>>>(part, splits, n, g);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Elementwise kernels.
// ---------------------------------------------------------------------------

// dz = dy * act'(y) (leaky ReLU, from the sign of the activation's output;
// identity when !act); also accumulates dz into skip_grad if given, and the
// per-channel sums over this block's pixels into bias_part[block][c].
__global__ void k_act_back(const float *__restrict__ dy, const bf16 *__restrict__ y, long long P,
                           int C, bool act, bf16 *__restrict__ dz, float *__restrict__ skip_grad,
                           float *__restrict__ bias_part, long long pix_per_block) {
    extern __shared__ float csum[];
    for (int c = threadIdx.x; c < C; c += blockDim.x) csum[c] = 0.f;
    __syncthreads();
    const long long p0 = blockIdx.x * pix_per_block;
    long long p1 = p0 + pix_per_block;
    if (p1 > P) p1 = P;
    // each thread owns one channel (C <= blockDim.x * k)
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float s = 0.f;
        for (long long p = p0; p < p1; ++p) {
            const long long i = p * C + c;
            float g = dy[i];
            if (act && __bfloat162float(y[i]) <= 0.f) g *= LEAK;
            dz[i] = __float2bfloat16_rn(g);
            if (skip_grad) skip_grad[i] += g;
            s += g;
        }
        csum[c] = s;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) bias_part[blockIdx.x * (long long)C + c] = csum[c];
}

cudaError_t act_back(const float *dy, const bf16 *y, long long P, int C, bool act, bf16 *dz,
                     float *skip_grad, float *bias_part, int blocks, cudaStream_t st) {
    const long long per = (P + blocks - 1) / blocks;
    k_act_back<<<blocks, 256, C * sizeof(float), st>>>(dy, y, P, C, act, dz, skip_grad, bias_part,
                                                       per);
    return cudaGetLastError();
}

// 2x2 average pooling, NHWC bf16.
__global__ void k_pool(const bf16 *__restrict__ in, int B, int H, int W, int C,
                       bf16 *__restrict__ out) {
    const int h = H / 2, w = W / 2;
    const long long n = (long long)B * h * w * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % C);
        const long long pix = i / C;
        const int x = int(pix % w), y = int((pix / w) % h), b = int(pix / ((long long)w * h));
        const long long base = (((long long)b * H + 2 * y) * W + 2 * x) * C + c;
        const float s = __bfloat162float(in[base]) + __bfloat162float(in[base + C]) +
                        __bfloat162float(in[base + (long long)W * C]) +
                        __bfloat162float(in[base + (long long)W * C + C]);
        out[i] = __float2bfloat16_rn(0.25f * s);
    }
}

// Gradient of the pooling: g_in[2y+a, 2x+b] += g_out[y, x] / 4 (fp32).
__global__ void k_pool_back(const float *__restrict__ gout, int B, int H, int W, int C,
                            float *__restrict__ gin) {
    const long long n = (long long)B * H * W * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % C);
        const long long pix = i / C;
        const int x = int(pix % W), y = int((pix / W) % H), b = int(pix / ((long long)W * H));
        gin[i] += 0.25f * gout[(((long long)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c];
    }
}

// Nearest-neighbour 2x upsampling, NHWC bf16.
__global__ void k_up(const bf16 *__restrict__ in, int B, int h, int w, int C,
                     bf16 *__restrict__ out) {
    const long long n = (long long)B * 4 * h * w * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % C);
        const long long pix = i / C;
        const int X = int(pix % (2 * w)), Y = int((pix / (2 * w)) % (2 * h));
        const int b = int(pix / (4LL * w * h));
        out[i] = in[(((long long)b * h + Y / 2) * w + X / 2) * C + c];
    }
}

// Gradient of the upsampling: g_in[y, x] = sum of the 4 g_out it fed (fp32).
__global__ void k_up_back(const float *__restrict__ gout, int B, int h, int w, int C,
                          float *__restrict__ gin) {
    const long long n = (long long)B * h * w * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % C);
        const long long pix = i / C;
        const int x = int(pix % w), y = int((pix / w) % h), b = int(pix / ((long long)w * h));
        const int W = 2 * w;
        const long long base = (((long long)b * 2 * h + 2 * y) * W + 2 * x) * C + c;
        gin[i] = gout[base] + gout[base + C] + gout[base + (long long)W * C] +
                 gout[base + (long long)W * C + C];
    }
}

// Flipped, transposed weights for the input gradient:
//   wt[ci][tap][co] = w[co][8 - tap][ci].
__global__ void k_flip(const bf16 *__restrict__ w, int cout, int cin, bf16 *__restrict__ wt) {
    const long long n = (long long)cout * 9 * cin;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int co = int(i % cout);
        const int tap = int((i / cout) % 9);
        const int ci = int(i / (9LL * cout));
        wt[i] = w[((long long)co * 9 + (8 - tap)) * cin + ci];
    }
}

// Adam on FP32 master weights; writes the BF16 copy the kernels use (wb may
// be null for parameters kept in FP32, the biases).
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2, bf16 *__restrict__ wb) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (wb) wb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_to_bf16(const float *__restrict__ a, long long n, bf16 *__restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

// Features (fp32 [P][FEAT]) -> padded bf16 input ([P][cpad], zeros beyond).
__global__ void k_pack_in(const float *__restrict__ f, long long P, int feat, int cpad,
                          bf16 *__restrict__ x) {
    const long long n = P * cpad;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % cpad);
        const long long p = i / cpad;
        x[i] = __float2bfloat16_rn(c < feat ? f[p * feat + c] : 0.f);
    }
}

// Loss: mean over pixels and the first `nout` channels of (y - t)^2;
// dy = 2 (y - t) / count there, 0 in the padded channels; per-block sums.
__global__ void k_mse(const float *__restrict__ y, int cpad, const float *__restrict__ t, int nout,
                      long long P, float *__restrict__ dy, double *__restrict__ part) {
    __shared__ double red[256];
    const double inv = 1.0 / double(P * nout);
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * cpad;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % cpad);
        const long long p = i / cpad;
        float g = 0.f;
        if (c < nout) {
            const float d = y[i] - t[p * nout + c];
            s += double(d) * d;
            g = float(2.0 * d * inv);
        }
        dy[i] = g;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0] * inv;
}

// out[p][c] = y[p][c] for c < nout (strip the padded channels).
__global__ void k_strip(const float *__restrict__ y, int cpad, int nout, long long P,
                        float *__restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * nout;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / nout;
        out[i] = y[p * cpad + int(i % nout)];
    }
}

int ew_blocks(long long n) { return int(std::min<long long>((n + 255) / 256, 8192)); }

}  // namespace surr
