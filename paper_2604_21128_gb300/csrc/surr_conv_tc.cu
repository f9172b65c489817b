// 3x3 periodic convolution of the learned surrogate on the fifth-generation
// tensor cores: an implicit GEMM
//   out[p, co] = sum_{tap, ci} w[co][tap][ci] * in[p shifted by tap, ci]
// with M = 128 pixels per CTA (one TMEM lane each), N = NT output channels,
// and K walked one tap and 32 input channels per pipeline stage.
//
// All 128 threads gather the stage's operands with cp.async into shared
// memory in the no-swizzle K-major layout of the UMMA descriptors (8-row x
// 16-byte core matrices, 128 bytes each; K-adjacent core matrices 128 bytes
// apart, 8-row groups 512 bytes apart).  One thread issues two
// tcgen05.mma (K = 16 each) per stage into an FP32 accumulator in TMEM and
// commits them to the stage's mbarrier, which frees the stage for the loads
// two stages later.  The epilogue reads the accumulator back with
// tcgen05.ld (warp w owns TMEM lanes 32w .. 32w + 31, i.e. its 32 pixels)
// and applies bias, skip, activation and the output conversion.
//
// Every wait on an mbarrier has an iteration limit; a CTA that gives up sets
// conv_tc_error, skips its epilogue, frees its TMEM and returns.
#include "surr_internal.h"

namespace surr {
namespace {

constexpr int TM = 128;          // pixels per CTA = TMEM lanes
constexpr int KC = 32;           // input channels per stage (two K = 16 MMAs)
constexpr int NSTAGE = 4;        // shared-memory stages
constexpr int AHEAD = NSTAGE - 2;  // stages loaded ahead of the MMA
constexpr unsigned WAIT_LIMIT = 1u << 22;

__device__ int g_conv_tc_error;

// Shared-memory matrix descriptor (tcgen05 format): start address, leading
// byte offset (K direction), stride byte offset (8-row direction), all in
// 16-byte units; descriptor version 1 at bit 46; no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at
// bit 17, M / 16 at bit 24.
template <int N>
__host__ __device__ constexpr uint32_t umma_idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) |
           (uint32_t(TM >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
    const uint32_t a = smem_u32(b);
    for (unsigned i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, one 128 x N x 16 step.
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the mbarrier once every MMA this thread issued so far is done.
__device__ __forceinline__ void umma_commit(uint64_t *b) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(b))
        : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int NT>
constexpr int stage_bytes() {
    return TM * KC * 2 + NT * KC * 2;
}

template <int NT, int MODE, bool ACT, bool SKIP>
__global__ void __launch_bounds__(128)
k_conv3x3_tc(const bf16 *__restrict__ in, int B, int H, int W, int cin,
             const bf16 *__restrict__ w, int cout, const float *__restrict__ bias,
             const bf16 *__restrict__ skip, bf16 *__restrict__ out_bf, float *__restrict__ out_f) {
    constexpr int A_BYTES = TM * KC * 2;
    constexpr int STAGE = stage_bytes<NT>();
    constexpr uint32_t TCOLS = NT;   // a power of two, >= 32
    static_assert(NT == 32 || NT == 64 || NT == 128 || NT == 256, "TMEM allocation size");
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[NSTAGE];
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5;
    const long long P = (long long)B * H * W;
    const long long p0 = (long long)blockIdx.x * TM;
    const int co0 = blockIdx.y * NT;

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&bar[s]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    // this thread's pixel (A row) and its place in the A tile
    const long long pa = p0 + tid;
    const bool a_ok = pa < P;
    int ab = 0, ay = 0, ax = 0;
    if (a_ok) {
        ab = int(pa / ((long long)H * W));
        const int rem = int(pa - (long long)ab * H * W);
        ay = rem / W;
        ax = rem - ay * W;
    }
    const uint32_t a_off = uint32_t((tid >> 3) * 4 * 128 + (tid & 7) * 16);
    const int kchunks = cin / KC;
    const int ksteps = 9 * kchunks;

    auto load = [&](int ks) {
        unsigned char *sa = smem + (ks % NSTAGE) * STAGE;
        unsigned char *sb = sa + A_BYTES;
        const int tap = ks / kchunks, ci0 = (ks - tap * kchunks) * KC;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        if (a_ok) {
            const long long ps = (long long)ab * H * W + (long long)wrapi(ay + dy, H) * W +
                                 wrapi(ax + dx, W);
            const bf16 *src = in + ps * cin + ci0;
#pragma unroll
            for (int kg = 0; kg < 4; ++kg) cp16(sa + a_off + kg * 128, src + kg * 8);
        } else {
#pragma unroll
            for (int kg = 0; kg < 4; ++kg)
                *reinterpret_cast<uint4 *>(sa + a_off + kg * 128) = make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int c = tid; c < NT * 4; c += 128) {
            const int n = c >> 2, kg = c & 3;
            cp16(sb + ((n >> 3) * 4 + kg) * 128 + (n & 7) * 16,
                 w + ((long long)(co0 + n) * 9 + tap) * cin + ci0 + kg * 8);
        }
    };

    bool ok = true;
#pragma unroll
    for (int i = 0; i < AHEAD; ++i) {
        if (i < ksteps) load(i);
        cp_commit();
    }
    for (int ks = 0; ks < ksteps; ++ks) {
        const int kn = ks + AHEAD;
        if (kn < ksteps) {
            // stage kn % NSTAGE last served step kn - NSTAGE; its MMAs must be done
            if (ok && kn >= NSTAGE) ok = mbar_wait(&bar[kn % NSTAGE], ((kn - NSTAGE) / NSTAGE) & 1);
            if (ok) load(kn);
        }
        cp_commit();
        cp_wait<AHEAD>();
        // this thread's copies (and zero fills) of step ks are in shared
        // memory; make them visible to the tensor core's async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && ok) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(smem + (ks % NSTAGE) * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
            for (int k = 0; k < KC / 16; ++k)
                umma(tmem, umma_desc(a0 + k * 256, 128, 512), umma_desc(b0 + k * 256, 128, 512),
                     umma_idesc<NT>(), (ks | k) != 0);
            umma_commit(&bar[ks % NSTAGE]);
        }
    }
    // the last commit covers every MMA of the tile
    if (ok) {
        const int kl = ksteps - 1;
        ok = mbar_wait(&bar[kl % NSTAGE], (kl / NSTAGE) & 1);
    }
    cp_wait<0>();
    // tcgen05.ld is warp-collective: every thread takes the same branch below
    ok = __syncthreads_and(ok);
    tc_fence_after();

    if (ok) {
        const uint32_t lane_base = tmem + (uint32_t(warp * 32) << 16);
        const long long p = pa;
#pragma unroll 1
        for (int c0 = 0; c0 < NT; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base + uint32_t(c0), v);
            if (p >= P) continue;
            const int co = co0 + c0;
            if constexpr (MODE == OUT_BF16) {
                if (bias) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += bias[co + i];
                }
                if constexpr (SKIP) {
                    const uint4 *s = reinterpret_cast<const uint4 *>(skip + p * cout + co);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint4 u = s[h];
                        const uint32_t wd[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            __nv_bfloat162 b2;
                            *reinterpret_cast<uint32_t *>(&b2) = wd[j];
                            v[h * 8 + 2 * j] += __bfloat162float(b2.x);
                            v[h * 8 + 2 * j + 1] += __bfloat162float(b2.y);
                        }
                    }
                }
                if constexpr (ACT) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = v[i] > 0.f ? v[i] : LEAK * v[i];
                }
                uint32_t wd[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                    wd[j] = *reinterpret_cast<const uint32_t *>(&b2);
                }
                uint4 *o = reinterpret_cast<uint4 *>(out_bf + p * cout + co);
                o[0] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                o[1] = make_uint4(wd[4], wd[5], wd[6], wd[7]);
            } else if constexpr (MODE == OUT_F32) {
                if (bias) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += bias[co + i];
                }
                float4 *o = reinterpret_cast<float4 *>(out_f + p * cout + co);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            } else {
                float4 *o = reinterpret_cast<float4 *>(out_f + p * cout + co);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 prev = o[j];
                    o[j] = make_float4(prev.x + v[4 * j], prev.y + v[4 * j + 1],
                                       prev.z + v[4 * j + 2], prev.w + v[4 * j + 3]);
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(&g_conv_tc_error, 1);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TCOLS)
                     : "memory");
}

template <int NT, int MODE, bool ACT, bool SKIP>
cudaError_t launch_nt(const ConvArgs &a, long long mtiles, cudaStream_t st) {
    auto k = k_conv3x3_tc<NT, MODE, ACT, SKIP>;
    constexpr int smem = NSTAGE * stage_bytes<NT>();
    static cudaError_t attr = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   smem);
    if (attr != cudaSuccess) return attr;
    k<<<dim3(unsigned(mtiles), unsigned(a.cout / NT)), 128, smem, st>>>(
        a.in, a.B, a.H, a.W, a.cin, a.w, a.cout, a.bias, a.skip, a.out_bf, a.out_f);
    return cudaGetLastError();
}

template <int MODE, bool ACT, bool SKIP>
cudaError_t conv_tc_t(const ConvArgs &a, cudaStream_t st) {
    const long long P = (long long)a.B * a.H * a.W;
    const long long mtiles = (P + TM - 1) / TM;
    // the widest N tile that divides cout and still gives about one CTA per SM
    int nt = 256;
    while (nt > 32 && (a.cout % nt != 0 || mtiles * (a.cout / nt) < 152)) nt >>= 1;
    switch (nt) {
    case 256: return launch_nt<256, MODE, ACT, SKIP>(a, mtiles, st);
    case 128: return launch_nt<128, MODE, ACT, SKIP>(a, mtiles, st);
    case 64: return launch_nt<64, MODE, ACT, SKIP>(a, mtiles, st);
    default: return launch_nt<32, MODE, ACT, SKIP>(a, mtiles, st);
    }
}

}  // namespace

cudaError_t conv3x3_tc(const ConvArgs &a, int mode, bool act, bool skip, cudaStream_t st) {
    if (a.cin % KC || a.cout % 32) return cudaErrorInvalidValue;
    if (mode == OUT_BF16) {
        if (act)
            return skip ? conv_tc_t<OUT_BF16, true, true>(a, st)
                        : conv_tc_t<OUT_BF16, true, false>(a, st);
        return skip ? conv_tc_t<OUT_BF16, false, true>(a, st)
                    : conv_tc_t<OUT_BF16, false, false>(a, st);
    }
    if (mode == OUT_F32) return conv_tc_t<OUT_F32, false, false>(a, st);
    return conv_tc_t<ACC_F32, false, false>(a, st);
}

cudaError_t conv_tc_error(int *flag, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(flag, g_conv_tc_error, sizeof(int));
    if (e == cudaSuccess && reset) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_conv_tc_error, &zero, sizeof(int));
    }
    return e;
}

}  // namespace surr
