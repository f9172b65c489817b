// Convolution kernels of the learned surrogate: the 3x3 periodic convolution
// (forward, and input gradient with flipped, transposed weights) runs on the
// tcgen05 tensor cores (surr_conv_tc.cu); here are the weight gradient as a
// split-K GEMM over the pixels (warp-level mma.sync) with a fixed-order
// reduction, and the elementwise kernels around them.  All tensors are NHWC;
// channel counts are multiples of 32.
#include "surr_internal.h"

namespace surr {

// ---------------------------------------------------------------------------
// Forward / input-gradient convolution: the tcgen05 implicit GEMM of
// surr_conv_tc.cu.  Epilogue by MODE:
//   OUT_BF16: out_bf = act(acc + bias + skip)   (act optional)
//   OUT_F32 : out_f  = acc + bias
//   ACC_F32 : out_f += acc
// ---------------------------------------------------------------------------
cudaError_t conv3x3(const ConvArgs &a, int mode, bool act, bool skip, cudaStream_t st) {
    if (a.cin % 32 || a.cout % 32) return cudaErrorInvalidValue;
    return conv3x3_tc(a, mode, act, skip, st);
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

// Many splits of few values (the per-block bias sums): one block per value,
// each thread a strided share of the splits, then a fixed-order tree.
__global__ void k_sum_splits_tree(const float *__restrict__ part, int splits, long long n,
                                  float *__restrict__ g) {
    __shared__ float red[256];
    const long long i = blockIdx.x;
    float s = 0.f;
    for (int k = threadIdx.x; k < splits; k += blockDim.x) s += part[k * n + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) g[i] = red[0];
}

cudaError_t sum_splits(const float *part, int splits, long long n, float *g, cudaStream_t st) {
    if (splits >= 64 && n <= 65535) {
        k_sum_splits_tree<<<unsigned(n), 256, 0, st>>>(part, splits, n, g);
    } else {
        const int blocks = int(std::min<long long>((n + 255) / 256, 4096));
        k_sum_splits<<<blocks, 256, 0, st>>>(part, splits, n, g);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Elementwise kernels.  Tensors are NHWC with C a multiple of 32; a thread
// handles eight BF16 or four FP32 channels of one pixel, and every index fits
// 32 bits (checked where the network is sized).
// ---------------------------------------------------------------------------

__device__ __forceinline__ void unpack8(uint4 u, float (&v)[8]) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        __nv_bfloat162 b;
        *reinterpret_cast<uint32_t *>(&b) = w[j];
        v[2 * j] = __bfloat162float(b.x);
        v[2 * j + 1] = __bfloat162float(b.y);
    }
}

__device__ __forceinline__ uint4 pack8(const float (&v)[8]) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        w[j] = *reinterpret_cast<const uint32_t *>(&b);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ uint4 ld8(const bf16 *p) { return *reinterpret_cast<const uint4 *>(p); }
__device__ __forceinline__ float4 ld4(const float *p) {
    return *reinterpret_cast<const float4 *>(p);
}

// dz = dy * act'(y) (leaky ReLU, from the sign of the activation's output;
// identity when !act); also accumulates dz into skip_grad if given, and the
// per-channel sums over this block's pixels into bias_part[block][c].
// Thread t takes channel t % C of every (256 / C)-th pixel; the phases are
// summed in a fixed order.
__global__ void k_act_back(const float *__restrict__ dy, const bf16 *__restrict__ y, long long P,
                           int C, bool act, bf16 *__restrict__ dz, float *__restrict__ skip_grad,
                           float *__restrict__ bias_part, long long pix_per_block) {
    __shared__ float red[256];
    const int R = blockDim.x / C;
    const int c = threadIdx.x % C, r = threadIdx.x / C;
    const long long p0 = blockIdx.x * pix_per_block;
    long long p1 = p0 + pix_per_block;
    if (p1 > P) p1 = P;
    float s = 0.f;
    for (long long p = p0 + r; p < p1; p += R) {
        const long long i = p * C + c;
        float g = dy[i];
        if (act && __bfloat162float(y[i]) <= 0.f) g *= LEAK;
        dz[i] = __float2bfloat16_rn(g);
        if (skip_grad) skip_grad[i] += g;
        s += g;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < C) {
        float t = 0.f;
        for (int k = 0; k < R; ++k) t += red[k * C + threadIdx.x];
        bias_part[blockIdx.x * (long long)C + threadIdx.x] = t;
    }
}

cudaError_t act_back(const float *dy, const bf16 *y, long long P, int C, bool act, bf16 *dz,
                     float *skip_grad, float *bias_part, int blocks, cudaStream_t st) {
    if (C > 256 || 256 % C) return cudaErrorInvalidValue;
    const long long per = (P + blocks - 1) / blocks;
    k_act_back<<<blocks, 256, 0, st>>>(dy, y, P, C, act, dz, skip_grad, bias_part, per);
    return cudaGetLastError();
}

// 2x2 average pooling, NHWC bf16.
__global__ void k_pool(const bf16 *__restrict__ in, int B, int H, int W, int C,
                       bf16 *__restrict__ out) {
    const unsigned h = H / 2, w = W / 2, c8n = C / 8;
    const unsigned n = unsigned(B) * h * w * c8n;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned c8 = i % c8n, pix = i / c8n;
        const unsigned x = pix % w, t = pix / w, y = t % h, b = t / h;
        const size_t base = ((size_t(b) * H + 2 * y) * W + 2 * x) * C + c8 * 8;
        const size_t row = size_t(W) * C;
        float a[8], bb[8], cc[8], d[8], o[8];
        unpack8(ld8(in + base), a);
        unpack8(ld8(in + base + C), bb);
        unpack8(ld8(in + base + row), cc);
        unpack8(ld8(in + base + row + C), d);
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = 0.25f * (a[j] + bb[j] + cc[j] + d[j]);
        *reinterpret_cast<uint4 *>(out + size_t(pix) * C + c8 * 8) = pack8(o);
    }
}

// Gradient of the pooling: g_in[2y+a, 2x+b] += g_out[y, x] / 4 (fp32).
__global__ void k_pool_back(const float *__restrict__ gout, int B, int H, int W, int C,
                            float *__restrict__ gin) {
    const unsigned c4n = C / 4;
    const unsigned n = unsigned(B) * H * W * c4n;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned c4 = i % c4n, pix = i / c4n;
        const unsigned x = pix % W, t = pix / W, y = t % H, b = t / H;
        const float4 g = ld4(gout + ((size_t(b) * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c4 * 4);
        float4 *o = reinterpret_cast<float4 *>(gin + size_t(pix) * C + c4 * 4);
        float4 v = *o;
        v.x += 0.25f * g.x;
        v.y += 0.25f * g.y;
        v.z += 0.25f * g.z;
        v.w += 0.25f * g.w;
        *o = v;
    }
}

// Nearest 2x upsampling, NHWC bf16.
__global__ void k_up(const bf16 *__restrict__ in, int B, int h, int w, int C,
                     bf16 *__restrict__ out) {
    const unsigned c8n = C / 8, W = 2 * w, H = 2 * h;
    const unsigned n = unsigned(B) * H * W * c8n;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned c8 = i % c8n, pix = i / c8n;
        const unsigned X = pix % W, t = pix / W, Y = t % H, b = t / H;
        *reinterpret_cast<uint4 *>(out + size_t(pix) * C + c8 * 8) =
            ld8(in + ((size_t(b) * h + Y / 2) * w + X / 2) * C + c8 * 8);
    }
}

// Gradient of the upsampling: g_in[y, x] = sum of the 4 g_out it fed (fp32).
__global__ void k_up_back(const float *__restrict__ gout, int B, int h, int w, int C,
                          float *__restrict__ gin) {
    const unsigned c4n = C / 4, W = 2 * w;
    const unsigned n = unsigned(B) * h * w * c4n;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned c4 = i % c4n, pix = i / c4n;
        const unsigned x = pix % w, t = pix / w, y = t % h, b = t / h;
        const size_t base = ((size_t(b) * 2 * h + 2 * y) * W + 2 * x) * C + c4 * 4;
        const size_t row = size_t(W) * C;
        const float4 a = ld4(gout + base), bb = ld4(gout + base + C), c = ld4(gout + base + row),
                     d = ld4(gout + base + row + C);
        *reinterpret_cast<float4 *>(gin + size_t(pix) * C + c4 * 4) =
            make_float4(a.x + bb.x + c.x + d.x, a.y + bb.y + c.y + d.y, a.z + bb.z + c.z + d.z,
                        a.w + bb.w + c.w + d.w);
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
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
         p += (long long)gridDim.x * blockDim.x) {
        for (int c0 = 0; c0 < cpad; c0 += 8) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = c0 + j < feat ? f[p * feat + c0 + j] : 0.f;
            *reinterpret_cast<uint4 *>(x + p * cpad + c0) = pack8(v);
        }
    }
}

// Loss: mean over pixels and the first `nout` channels of (y - t)^2;
// dy = 2 (y - t) / count there, 0 in the padded channels; per-block sums.
__global__ void k_mse(const float *__restrict__ y, int cpad, const float *__restrict__ t, int nout,
                      long long P, float *__restrict__ dy, double *__restrict__ part) {
    __shared__ double red[256];
    const double inv = 1.0 / double(P * nout);
    double s = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
         p += (long long)gridDim.x * blockDim.x) {
        for (int c0 = 0; c0 < cpad; c0 += 4) {
            float g[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                g[j] = 0.f;
                if (c0 + j < nout) {
                    const float d = y[p * cpad + c0 + j] - t[p * nout + c0 + j];
                    s += double(d) * d;
                    g[j] = float(2.0 * d * inv);
                }
            }
            *reinterpret_cast<float4 *>(dy + p * cpad + c0) = make_float4(g[0], g[1], g[2], g[3]);
        }
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
