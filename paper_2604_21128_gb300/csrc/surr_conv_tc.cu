// 3x3 periodic convolution of the learned surrogate on the fifth-generation
// tensor cores: an implicit GEMM
//   out[p, co] = sum_{tap, ci} w[co][tap][ci] * in[p shifted by tap, ci]
// with M = 128 pixels per CTA (one TMEM lane each), N = NT output channels,
// and K walked in 32-channel chunks.
//
// Operands sit in shared memory in the no-swizzle K-major layout of the UMMA
// descriptors (8-row x 16-byte core matrices).  One thread issues the
// tcgen05.mma (K = 16 each) into an FP32 accumulator in TMEM and commits them
// to an mbarrier, which frees their shared memory for later loads.  The
// epilogue reads the accumulator back with tcgen05.ld (warp w owns TMEM lanes
// 32w .. 32w + 31, i.e. its 32 pixels) and applies bias, skip, activation and
// the output conversion.
//
// Two kernels: k_conv3x3_tc gathers a stage per tap and 32 or 64 channels
// (six or four stages, two fewer loaded ahead); k_conv3x3_rows, for widths
// that are multiples of 128,
// loads one halo'd row patch per chunk that serves all nine taps and keeps
// the weights resident in persistent CTAs.
//
// Every wait on an mbarrier gives up after WAIT_NS of %globaltimer time; a CTA
// that gives up sets conv_tc_error, skips its epilogue, frees its TMEM and
// returns.  After such a timeout the launch's outputs are undefined, and so is
// the TMEM it freed if the wait that ran out was on MMAs still in flight (a
// genuine hang of the tensor pipe rather than a phase that never comes): the
// caller should rebuild the network before trusting another result.
#include <cuda.h>

#include "surr_internal.h"

namespace surr {
namespace {

constexpr int TM = 128;          // pixels per CTA = TMEM lanes
constexpr int KC = 32;           // input channels per row-patch chunk (two K = 16 MMAs)

// Gather-kernel stages: KS input channels of one tap (KS / 16 MMAs), six
// stages of 32 channels or four of 64, all but two loaded ahead of the MMA.
template <int KS> constexpr int gather_stages() { return KS == 32 ? 6 : 4; }
constexpr unsigned long long WAIT_NS = 2000000000ull;   // a wait gives up after 2 s

__device__ int g_conv_tc_error;
// Test hook (surr_test_stall_conv): CTA (0, 0) of each launch waits for a
// phase that never completes, so its bounded wait runs out.
__device__ int g_conv_tc_stall;

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

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity; false once WAIT_NS of wall time
// have passed (try_wait may suspend the thread for a while on each call, so
// the bound is on time, not on the number of calls).
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
    const uint32_t a = smem_u32(b);
    if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try(a, parity)) return true;
        if (global_ns() - t0 > WAIT_NS) return false;
    }
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

// The accumulator rows of this thread's TMEM lane (lane_base) -> output
// pixel p, channels co0 .. co0 + NT - 1, by MODE (see conv3x3).  Every thread
// of the warp takes part in the loads; only valid pixels store.
template <int NT, int MODE, bool ACT, bool SKIP>
__device__ __forceinline__ void epilogue(uint32_t lane_base, long long p, bool valid, int co0,
                                         int cout, const float *__restrict__ bias,
                                         const bf16 *__restrict__ skip, bf16 *__restrict__ out_bf,
                                         float *__restrict__ out_f) {
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += 16) {
        float v[16];
        tmem_ld16(lane_base + uint32_t(c0), v);
        if (!valid) continue;
        const int co = co0 + c0;
        if constexpr (MODE == OUT_BF16) {
            if (bias) {
                const float4 *bb = reinterpret_cast<const float4 *>(bias + co);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 t = bb[j];
                    v[4 * j] += t.x;
                    v[4 * j + 1] += t.y;
                    v[4 * j + 2] += t.z;
                    v[4 * j + 3] += t.w;
                }
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
                const float4 *bb = reinterpret_cast<const float4 *>(bias + co);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 t = bb[j];
                    v[4 * j] += t.x;
                    v[4 * j + 1] += t.y;
                    v[4 * j + 2] += t.z;
                    v[4 * j + 3] += t.w;
                }
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
}

template <int NT, int KS>
constexpr int stage_bytes() {
    return TM * KS * 2 + NT * KS * 2;
}

template <int NT, int KS, int MODE, bool ACT, bool SKIP>
__global__ void __launch_bounds__(128)
k_conv3x3_tc(const bf16 *__restrict__ in, int B, int H, int W, int cin,
             const bf16 *__restrict__ w, int cout, const float *__restrict__ bias,
             const bf16 *__restrict__ skip, bf16 *__restrict__ out_bf, float *__restrict__ out_f) {
    constexpr int NSTAGE = gather_stages<KS>(), AHEAD = NSTAGE - 2;
    constexpr int KG = KS / 8;                 // 16-byte channel groups per stage
    constexpr int A_BYTES = TM * KS * 2;
    constexpr int STAGE = stage_bytes<NT, KS>();
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
    const uint32_t a_off = uint32_t((tid >> 3) * KG * 128 + (tid & 7) * 16);
    const int kchunks = cin / KS;
    const int ksteps = 9 * kchunks;

    auto load = [&](int ks) {
        unsigned char *sa = smem + (ks % NSTAGE) * STAGE;
        unsigned char *sb = sa + A_BYTES;
        const int tap = ks / kchunks, ci0 = (ks - tap * kchunks) * KS;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        if (a_ok) {
            const long long ps = (long long)ab * H * W + (long long)wrapi(ay + dy, H) * W +
                                 wrapi(ax + dx, W);
            const bf16 *src = in + ps * cin + ci0;
#pragma unroll
            for (int kg = 0; kg < KG; ++kg) cp16(sa + a_off + kg * 128, src + kg * 8);
        } else {
#pragma unroll
            for (int kg = 0; kg < KG; ++kg)
                *reinterpret_cast<uint4 *>(sa + a_off + kg * 128) = make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int c = tid; c < NT * KG; c += 128) {
            const int n = c / KG, kg = c % KG;
            cp16(sb + ((n >> 3) * KG + kg) * 128 + (n & 7) * 16,
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
            for (int k = 0; k < KS / 16; ++k)
                umma(tmem, umma_desc(a0 + k * 256, 128, KG * 128),
                     umma_desc(b0 + k * 256, 128, KG * 128),
                     umma_idesc<NT>(), (ks | k) != 0);
            umma_commit(&bar[ks % NSTAGE]);
        }
    }
    // the last commit covers every MMA of the tile
    if (ok) {
        const int kl = ksteps - 1;
        // the test hook waits for the phase after the last one (never completes)
        const uint32_t stall = g_conv_tc_stall && blockIdx.x == 0 && blockIdx.y == 0;
        ok = mbar_wait(&bar[kl % NSTAGE], ((kl / NSTAGE) & 1) ^ stall);
    }
    cp_wait<0>();
    // tcgen05.ld is warp-collective: every thread takes the same branch below
    ok = __syncthreads_and(ok);
    tc_fence_after();

    if (ok) {
        epilogue<NT, MODE, ACT, SKIP>(tmem + (uint32_t(warp * 32) << 16), pa, pa < P, co0, cout,
                                      bias, skip, out_bf, out_f);
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

// ---------------------------------------------------------------------------
// Row-patch variant for W a multiple of 128: a tile is 128 consecutive pixels
// of one image row, so every tap's operand is the same row patch shifted.  Per
// 32-channel chunk the CTA loads the patch once -- rows y-1, y, y+1 of pixels
// x0-1 .. x0+128 (periodic) -- laid out as [row][8-channel group][pixel][16
// bytes], i.e. K-major core matrices with 8-row groups 128 bytes apart (SBO)
// and channel groups PATCH_ARR bytes apart (LBO).  Tap (dy, dx) is then the
// descriptor whose start is row dy + 1, pixel dx + 1: 18 MMAs per chunk
// (9 taps x K = 32) read one patch.
//
// The patch's 128 interior pixels of each row and channel group arrive by
// TMA (cp.async.bulk.tensor over the NHWC activations, box 8 channels x 128
// pixels, 2 KB, 128-byte aligned in shared memory), twelve copies per patch
// issued by one thread and counted on the buffer's "full" mbarrier; the two
// wrapped edge pixels of each row and group come by cp.async.
//
// CTAs are persistent over the tiles and keep their N-slice of the weights in
// shared memory for the whole launch ([tap][chunk][channel group][n][16
// bytes]), so the weights leave L2 once per CTA instead of once per tile.
// Patches rotate through PATCH_BUF buffers: item i + PATCH_BUF - 1 loads while
// item i's MMAs run, once the MMAs of item i - 1 (which read that buffer) are
// done.  After a tile's last chunk the CTA waits for its MMAs and runs the
// epilogue from TMEM.
// ---------------------------------------------------------------------------
constexpr int PATCH_ARR = 2304;                  // bytes per [row][group] array (18 x 128)
constexpr int PATCH_BUF = 2;                     // patch buffers per CTA
constexpr int PATCH_J0 = 112;                    // offset of pixel 0: pixel 1 is 128-aligned
constexpr int PATCH_BYTES = 3 * 4 * PATCH_ARR;   // 3 rows x 4 channel groups
constexpr uint32_t PATCH_TMA_BYTES = 12 * TM * 16;

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}

// 4-D tiled TMA load (channels, x, y, image) into shared memory, completing
// on the mbarrier's transaction count.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c, int x,
                                            int y, int b, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(x), "r"(y), "r"(b), "r"(smem_u32(bar))
        : "memory");
}

template <int NT, int MODE, bool ACT, bool SKIP>
__global__ void __launch_bounds__(128)
k_conv3x3_rows(const __grid_constant__ CUtensorMap tmap, const bf16 *__restrict__ in, int B,
               int H, int W, int cin, const bf16 *__restrict__ w, int cout,
               const float *__restrict__ bias, const bf16 *__restrict__ skip,
               bf16 *__restrict__ out_bf, float *__restrict__ out_f) {
    constexpr int nbuf = PATCH_BUF;
    constexpr uint32_t TCOLS = NT;
    static_assert(NT == 32 || NT == 64 || NT == 128 || NT == 256, "TMEM allocation size");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mma_done[PATCH_BUF];
    __shared__ __align__(8) uint64_t full[PATCH_BUF];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int co0 = blockIdx.y * NT;
    const int kchunks = cin / KC;
    const long long P = (long long)B * H * W;
    const long long ntiles = P / TM;
    // this CTA's tiles: blockIdx.x, + gridDim.x, ...
    const long long my_tiles =
        blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long nitems = my_tiles * kchunks;
    // TMA destinations must be 128-byte aligned: align the base (the launch
    // adds 128 bytes of slack)
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    unsigned char *wsm = smem;                                   // weights
    unsigned char *patch = smem + size_t(18) * cin * NT;         // nbuf patch buffers

    if (tid == 0) {
        for (int k = 0; k < nbuf; ++k) {
            mbar_init(&mma_done[k]);
            mbar_init(&full[k]);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
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

    // weights of output channels co0 .. co0 + NT - 1, all taps and chunks
    {
        const int ci8n = cin / 8;
        const int total = NT * 9 * ci8n;
        for (int q = tid; q < total; q += 128) {
            const int ci8 = q % ci8n, t = (q / ci8n) % 9, n = q / (ci8n * 9);
            const int c = ci8 >> 2, kg = ci8 & 3;
            cp16(wsm + ((size_t(t * kchunks + c) * 4 + kg) * NT + n) * 16,
                 w + ((long long)(co0 + n) * 9 + t) * cin + ci8 * 8);
        }
    }
    // threads 0 .. 23 write a patch buffer (thread 0 by TMA, all 24 an edge
    // pixel each); the rest only read it.  Pixel indices fit 32 bits (the
    // network's workspace check).
    auto load_patch = [&](unsigned tile, int c, int sb) {
        unsigned char *buf = patch + sb * PATCH_BYTES;
        const unsigned p0 = tile * unsigned(TM);
        const unsigned row = p0 / unsigned(W);       // b * H + y
        const int x0 = int(p0 - row * unsigned(W)), y = int(row % unsigned(H));
        const int b = int(row / unsigned(H));
        const int ym = y == 0 ? H - 1 : y - 1, yp = y == H - 1 ? 0 : y + 1;
        if (tid == 0) {
            mbar_expect_tx(&full[sb], PATCH_TMA_BYTES);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int yy = r == 0 ? ym : (r == 1 ? y : yp);
#pragma unroll
                for (int kg = 0; kg < 4; ++kg)
                    tma_load_4d(smem_u32(buf + (r * 4 + kg) * PATCH_ARR + PATCH_J0 + 16), &tmap,
                                c * KC + kg * 8, x0, yy, b, &full[sb]);
            }
        }
        const int r = tid >> 3, e = (tid >> 2) & 1, kg = tid & 3;
        const int yy = r == 0 ? ym : (r == 1 ? y : yp);
        const int xx = e ? (x0 + TM == W ? 0 : x0 + TM) : (x0 == 0 ? W - 1 : x0 - 1);
        cp16(buf + (r * 4 + kg) * PATCH_ARR + PATCH_J0 + (e ? (TM + 1) * 16 : 0),
             in + ((size_t(b) * H + yy) * W + xx) * cin + c * KC + kg * 8);
    };
    // items are (tile, chunk) pairs, chunk fastest; the tiles of this CTA are
    // blockIdx.x, + gridDim.x, ...
    auto advance = [&](unsigned &tile, int &c) {
        if (++c == kchunks) {
            c = 0;
            tile += gridDim.x;
        }
    };

    bool ok = true;
    unsigned pf_tile = blockIdx.x;   // next item to load
    int pf_c = 0;
    for (int k = 0; k < nbuf - 1; ++k) {
        if (k < nitems) {
            if (tid < 24) load_patch(pf_tile, pf_c, k % nbuf);
            advance(pf_tile, pf_c);
        }
        cp_commit();
    }
    unsigned cur_tile = blockIdx.x;
    int c = 0;
    for (long long i = 0; i < nitems; ++i) {
        const int sb = int(i % nbuf);
        if (ok && !mbar_wait(&full[sb], uint32_t(i / nbuf) & 1)) ok = false;
        cp_wait<PATCH_BUF - 2>();   // this item's edge pixels (later items' may fly)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        if (__syncthreads_or(!ok)) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t pb = smem_u32(patch + sb * PATCH_BYTES), wb = smem_u32(wsm);
#pragma unroll 1
            for (int t = 0; t < 9; ++t) {
                const int dy = t / 3, dx = t % 3;   // patch row, pixel offset
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t a = pb + (dy * 4 + 2 * h) * PATCH_ARR + PATCH_J0 + dx * 16;
                    const uint32_t bw = wb + ((t * kchunks + c) * 4 + 2 * h) * NT * 16;
                    umma(tmem, umma_desc(a, PATCH_ARR, 128), umma_desc(bw, NT * 16, 128),
                         umma_idesc<NT>(), (c | t | h) != 0);
                }
            }
            umma_commit(&mma_done[sb]);
        }
        if (i + nbuf - 1 < nitems) {
            if (tid < 24) {
                // the buffer of item i + nbuf - 1 last served item i - 1
                if (i >= 1 && !mbar_wait(&mma_done[(i - 1) % nbuf], uint32_t((i - 1) / nbuf) & 1))
                    ok = false;
                if (ok) load_patch(pf_tile, pf_c, int((i + nbuf - 1) % nbuf));
            }
            advance(pf_tile, pf_c);
        }
        cp_commit();
        if (c == kchunks - 1) {
            if (!mbar_wait(&mma_done[sb], uint32_t(i / nbuf) & 1)) ok = false;
            // tcgen05.ld is warp-collective: decide for the whole CTA
            if (__syncthreads_or(!ok)) break;
            tc_fence_after();
            const long long p = (long long)cur_tile * TM + tid;
            epilogue<NT, MODE, ACT, SKIP>(tmem + (uint32_t(warp * 32) << 16), p, true, co0, cout,
                                          bias, skip, out_bf, out_f);
        }
        advance(cur_tile, c);
    }
    cp_wait<0>();
    if (!ok) abort_flag = 1;
    tc_fence_before();
    __syncthreads();
    if (abort_flag) {
        // TMA copies may still be in flight: let them land (bounded) before
        // the CTA's shared memory is released
        if (tid == 0) {
            atomicExch(&g_conv_tc_error, 1);
            for (long long i = nitems - nbuf; i < nitems; ++i)
                if (i >= 0) mbar_wait(&full[i % nbuf], uint32_t(i / nbuf) & 1);
        }
        __syncthreads();
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TCOLS)
                     : "memory");
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime.
EncodeTiled encode_tiled() {
    static EncodeTiled fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return EncodeTiled(nullptr);
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

template <int NT, int MODE, bool ACT, bool SKIP>
cudaError_t launch_rows(const ConvArgs &a, long long ntiles, cudaStream_t st) {
    auto k = k_conv3x3_rows<NT, MODE, ACT, SKIP>;
    // TMA view of the input: (channels, x, y, image), box 8 channels x 128 pixels
    const EncodeTiled enc = encode_tiled();
    if (!enc || (reinterpret_cast<uintptr_t>(a.in) & 15)) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[4] = {cuuint64_t(a.cin), cuuint64_t(a.W), cuuint64_t(a.H),
                                cuuint64_t(a.B)};
    const cuuint64_t strides[3] = {cuuint64_t(a.cin) * 2, cuuint64_t(a.W) * a.cin * 2,
                                   cuuint64_t(a.H) * a.W * a.cin * 2};
    const cuuint32_t box[4] = {8, TM, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(a.in), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    // the device's SM count and shared-memory limits, read once (thread-safe)
    struct Dev { int sms, smem, smem_block; };
    static const Dev dv = [] {
        Dev d{0, 0, 0};
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&d.smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&d.smem_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (d.sms < 1) d.sms = 1;
        return d;
    }();
    const int dev_sms = dv.sms, dev_smem = dv.smem, dev_smem_block = dv.smem_block;
    // CTAs per SM from shared memory -- dynamic + static + the 1 KB the system
    // reserves per CTA -- and TMEM, 512 columns.  (Deeper patch rings measured
    // slower: the chunk's 18 MMAs into one accumulator, not the loads, bound
    // a CTA that has to give up CTAs per SM for them.)
    const int smem = 128 + 18 * a.cin * NT + PATCH_BUF * PATCH_BYTES;
    const int per_sm = std::min(std::min(dev_smem / (smem + 1024 + 256), 512 / NT), 16);
    if (smem > dev_smem_block || per_sm < 1) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 int(cudaSharedmemCarveoutMaxShared));
    if (e != cudaSuccess) return e;
    const int ny = a.cout / NT;
    long long ctas = (long long)dev_sms * per_sm / ny;
    if (ctas < 1) ctas = 1;
    if (ctas > ntiles) ctas = ntiles;
    k<<<dim3(unsigned(ctas), unsigned(ny)), 128, smem, st>>>(
        map, a.in, a.B, a.H, a.W, a.cin, a.w, a.cout, a.bias, a.skip, a.out_bf, a.out_f);
    return cudaGetLastError();
}

template <int NT, int KS, int MODE, bool ACT, bool SKIP>
cudaError_t launch_ks(const ConvArgs &a, long long mtiles, cudaStream_t st) {
    auto k = k_conv3x3_tc<NT, KS, MODE, ACT, SKIP>;
    constexpr int smem = gather_stages<KS>() * stage_bytes<NT, KS>();
    static cudaError_t attr = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   smem);
    if (attr != cudaSuccess) return attr;
    k<<<dim3(unsigned(mtiles), unsigned(a.cout / NT)), 128, smem, st>>>(
        a.in, a.B, a.H, a.W, a.cin, a.w, a.cout, a.bias, a.skip, a.out_bf, a.out_f);
    return cudaGetLastError();
}

// 64-channel stages (four MMAs per barrier) where the input channels allow.
template <int NT, int MODE, bool ACT, bool SKIP>
cudaError_t launch_nt(const ConvArgs &a, long long mtiles, cudaStream_t st) {
    return a.cin % 64 == 0 ? launch_ks<NT, 64, MODE, ACT, SKIP>(a, mtiles, st)
                           : launch_ks<NT, 32, MODE, ACT, SKIP>(a, mtiles, st);
}

// Streaming multiprocessors of the current device (1 if the query fails).
int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
        return 1;
    return n;
}

template <int MODE, bool ACT, bool SKIP>
cudaError_t conv_tc_t(const ConvArgs &a, cudaStream_t st) {
    const long long P = (long long)a.B * a.H * a.W;
    const long long mtiles = (P + TM - 1) / TM;
    if (a.W % TM == 0) {
        // row patches; the N slice whose weights fit in about 160 KB (the
        // 128^2 decoder layer, 128 -> 64 channels: N = 64 on 152 CTAs 94 us
        // against N = 32 on 76 x 2 CTAs 152 us, the limit at 100 KB)
        int nt = a.cout < 256 ? a.cout : 256;
        while (nt > 32 && (a.cout % nt != 0 || 18 * a.cin * nt > 160 * 1024)) nt >>= 1;
        if (18 * a.cin * nt <= 160 * 1024 && a.cout % nt == 0) {
            switch (nt) {
            case 256: return launch_rows<256, MODE, ACT, SKIP>(a, mtiles, st);
            case 128: return launch_rows<128, MODE, ACT, SKIP>(a, mtiles, st);
            case 64: return launch_rows<64, MODE, ACT, SKIP>(a, mtiles, st);
            default: return launch_rows<32, MODE, ACT, SKIP>(a, mtiles, st);
            }
        }
    }
    // the widest N tile that divides cout and still gives about one CTA per SM
    const long long sms = sm_count();
    int nt = 256;
    while (nt > 32 && (a.cout % nt != 0 || mtiles * (a.cout / nt) < sms)) nt >>= 1;
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

cudaError_t conv_tc_stall(int on) {
    return cudaMemcpyToSymbol(g_conv_tc_stall, &on, sizeof(int));
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
