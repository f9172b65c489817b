// Marching QLA step kernel: one step of Eq. 2e14 per launch, state and
// coefficients in registers, no shared memory.
//
// Each warp owns a window of 32*LX columns (LX consecutive columns per lane)
// and marches down a segment of rows.  The window overlaps its neighbours by
// 4 columns on each side: U_x reaches four cells along x (four of its eight
// collision layers pair neighbouring sites), so the outer 4 columns of each
// side are recomputed halo and only the inner 32*LX - 8 columns are stored.
//
// Row by row:
//  * U_x (Eq. 2e6) acts on the whole row in registers.  Its eight layers are
//    disjoint 2x2 rotations (see layer_of); a bond that crosses a lane
//    boundary is computed by the lane that owns the bond's site, after one
//    shuffle brings the partner value in and one sends the result back.
//  * U_y (Eq. 2e9) runs as a software pipeline along y.  A layer that pairs
//    site j with j-1 or j+1 can finish row r-1 only when row r arrives, so
//    each of the four neighbour layers delays its output by one row and
//    carries two values per pair and column.  The output row of U_y is four
//    rows behind the input row, with no y-halo to recompute.
//  * V_x, V_y (Eqs. 2e11-2e13) of a step are applied when its output row
//    next enters a launch (before U_x), so the stored buffer holds
//    U_y U_x Q and the sequence of operations on the data is that of Eq. 2e14;
//    read-outs apply the pending V (see qla_ctx::pending_v).  Planes that U_y
//    does not touch are stored right after U_x, the others four rows later.
// The collision coefficients of the four rows in flight sit in a register
// ring; records come from the medium table through a 4-byte index per site.
// The next row's state and records and the indices two rows ahead are loaded
// one iteration early.  The march loop is unrolled by four so that every ring
// slot is a fixed register.
#include "qla_internal.h"

namespace qla {
namespace {

constexpr int WARPS = 4;           // independent warps per CTA
constexpr int LAG = 4;             // rows between U_y input and output

template <typename T, int LX> struct Vec;
template <> struct Vec<float, 4> { using type = float4; };
template <> struct Vec<float, 2> { using type = float2; };
template <> struct Vec<double, 2> { using type = double2; };

// Streamed data (state planes, index rows) is read through L2 only, so that
// L1 keeps the medium records, which every row looks up.
template <typename T, int LX>
__device__ __forceinline__ void vload(const T *p, T (&v)[LX]) {
    const auto t = __ldcg(reinterpret_cast<const typename Vec<T, LX>::type *>(p));
    if constexpr (LX == 4) { v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
    else { v[0] = t.x; v[1] = t.y; }
}

template <typename T, int LX>
__device__ __forceinline__ void vstore(T *p, const T (&v)[LX]) {
    typename Vec<T, LX>::type t;
    if constexpr (LX == 4) { t.x = v[0]; t.y = v[1]; t.z = v[2]; t.w = v[3]; }
    else { t.x = v[0]; t.y = v[1]; }
    *reinterpret_cast<typename Vec<T, LX>::type *>(p) = t;
}

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_dn1(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// Rotate the bond (unmoved u, moved m) of a pair whose first component (the
// row holding cos, -g sin) is the moved one iff a_moved.
template <typename T, typename K>
__device__ __forceinline__ void bond_rot(T &u, T &m, K k, T g, bool a_moved) {
    if (a_moved) rotate(m, u, k, g);
    else rotate(u, m, k, g);
}

// Collision sign of layer L: C_x by +theta, C_y by -theta; adjoint flips.
template <bool XDIR, int L>
__device__ constexpr int layer_sign() {
    return (layer_of(L).dag ? -1 : 1) * (XDIR ? 1 : -1);
}

// ---------------------------------------------------------------------------
// U_x on one row.  q[c][x]: amplitude c at the lane's column x (absent
// planes are never touched); k[x]: the row's collision coefficients.
// ---------------------------------------------------------------------------
template <typename T, int P, int LX, int L>
__device__ __forceinline__ void ux_layer(T (&q)[6][LX], const typename Coef<T>::C (&k)[LX]) {
    constexpr Layer ly = layer_of(L);
    const T g = T(layer_sign<true, L>());
#pragma unroll
    for (int pk = 0; pk < 2; ++pk) {
        const Pair pr = pair_of(true, pk);
        if (plane_of<P>(pr.a) < 0) continue;
        if (ly.mover == 0) {
#pragma unroll
            for (int x = 0; x < LX; ++x) rotate(q[pr.a][x], q[pr.b][x], k[x], g);
            continue;
        }
        // moved / unmoved component of this pair in this layer
        const bool a_moved = (ly.mover == 1) == pr.a_is_m1;
        const int cm = a_moved ? pr.a : pr.b, cu = a_moved ? pr.b : pr.a;
        if (ly.shift < 0) {
            // bond at site x pairs u[x] with m[x-1]; the lane's first bond
            // takes m from the left lane and returns the result to it
            T mL = shfl_up1(q[cm][LX - 1]);
#pragma unroll
            for (int x = LX - 1; x >= 1; --x) bond_rot(q[cu][x], q[cm][x - 1], k[x], g, a_moved);
            bond_rot(q[cu][0], mL, k[0], g, a_moved);
            q[cm][LX - 1] = shfl_dn1(mL);
        } else {
            // bond at site x pairs u[x] with m[x+1]; the lane's last bond
            // takes m from the right lane and returns the result to it
            T mR = shfl_dn1(q[cm][0]);
#pragma unroll
            for (int x = 0; x < LX - 1; ++x) bond_rot(q[cu][x], q[cm][x + 1], k[x], g, a_moved);
            bond_rot(q[cu][LX - 1], mR, k[LX - 1], g, a_moved);
            q[cm][0] = shfl_up1(mR);
        }
    }
}

template <typename T, int P, int LX>
__device__ __forceinline__ void apply_ux(T (&q)[6][LX], const typename Coef<T>::C (&k)[LX]) {
    ux_layer<T, P, LX, 0>(q, k);
    ux_layer<T, P, LX, 1>(q, k);
    ux_layer<T, P, LX, 2>(q, k);
    ux_layer<T, P, LX, 3>(q, k);
    ux_layer<T, P, LX, 4>(q, k);
    ux_layer<T, P, LX, 5>(q, k);
    ux_layer<T, P, LX, 6>(q, k);
    ux_layer<T, P, LX, 7>(q, k);
}

// ---------------------------------------------------------------------------
// U_y pipeline stages.  q holds the row entering the stage; on return it
// holds the row leaving it (one row later for a neighbour layer).
// carry[L/2][pair][0..1][x]: the values a neighbour layer keeps between rows.
// ---------------------------------------------------------------------------
template <typename T, int P, int LX, int L>
__device__ __forceinline__ void uy_local(T (&q)[6][LX], const typename Coef<T>::C (&k)[LX]) {
    const T g = T(layer_sign<false, L>());
#pragma unroll
    for (int pk = 0; pk < 2; ++pk) {
        const Pair pr = pair_of(false, pk);
        if (plane_of<P>(pr.a) < 0) continue;
#pragma unroll
        for (int x = 0; x < LX; ++x) rotate(q[pr.a][x], q[pr.b][x], k[x], g);
    }
}

// k: coefficients of the bond site (the entering row for shift -1, the row
// before it for shift +1).
template <typename T, int P, int LX, int L>
__device__ __forceinline__ void uy_neighbour(T (&q)[6][LX], T (&carry)[2][2][LX],
                                             const typename Coef<T>::C (&k)[LX]) {
    constexpr Layer ly = layer_of(L);
    const T g = T(layer_sign<false, L>());
#pragma unroll
    for (int pk = 0; pk < 2; ++pk) {
        const Pair pr = pair_of(false, pk);
        if (plane_of<P>(pr.a) < 0) continue;
        const bool a_moved = (ly.mover == 1) == pr.a_is_m1;
        const int cm = a_moved ? pr.a : pr.b, cu = a_moved ? pr.b : pr.a;
#pragma unroll
        for (int x = 0; x < LX; ++x) {
            T &c0 = carry[pk][0][x], &c1 = carry[pk][1][x];
            const T u = q[cu][x], m = q[cm][x];
            if (ly.shift < 0) {
                // bond at this row r: (u_r, m_{r-1}); c0 = m_{r-1} before the
                // layer, c1 = u_{r-1} after it
                T uu = u, mm = c0;
                bond_rot(uu, mm, k[x], g, a_moved);
                q[cu][x] = c1;
                q[cm][x] = mm;
                c0 = m;
                c1 = uu;
            } else {
                // bond at row r-1: (u_{r-1}, m_r); c0 = u_{r-1} before the
                // layer, c1 = m_{r-1} after it
                T uu = c0, mm = m;
                bond_rot(uu, mm, k[x], g, a_moved);
                q[cu][x] = uu;
                q[cm][x] = c1;
                c0 = u;
                c1 = mm;
            }
        }
    }
}

template <int P> __device__ constexpr bool in_y_pair(int c) {
    return plane_of<P>(c) >= 0 && (c == 0 || c == 2 || c == 3 || c == 5);
}

// ---------------------------------------------------------------------------
// The kernel.  Work item = (window wx, row segment wy); one warp per item.
// ---------------------------------------------------------------------------
template <typename T, int LX> struct IdxVec;
template <> struct IdxVec<float, 4> { using type = uint4; };
template <> struct IdxVec<float, 2> { using type = uint2; };
template <> struct IdxVec<double, 2> { using type = uint2; };

template <typename T, int LX>
__device__ __forceinline__ void iload(const uint32_t *p, uint32_t (&v)[LX]) {
    const auto t = __ldcg(reinterpret_cast<const typename IdxVec<T, LX>::type *>(p));
    if constexpr (LX == 4) { v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
    else { v[0] = t.x; v[1] = t.y; }
}

template <typename T, int P, int LX, int VM, bool VIN>
struct March {
    using CC = typename Coef<T>::C;
    using CV = typename Coef<T>::V;
    static constexpr int W = 32 * LX;   // window columns
    static constexpr int WOUT = W - 8;  // stored columns

    const T *in;
    T *out;
    const uint32_t *midx;
    const MedRec<T> *table;
    int nx, ny, pitch, seg_h, n_wx, n_items;
    size_t plane;

    // state carried along the march
    T carry[4][2][2][LX];   // [neighbour layer][pair][value][x]
    CC kring[LAG][LX];      // collision coefficients of the rows in flight
    T qbuf[2][6][LX];       // this row and the prefetched next row (by parity)
    uint32_t ibuf[2][LX];   // record indices of rows J (parity of J) and J+1
    CC knext[LX];           // row J+1's records, looked up one row early
    CV vnext[LX];
    // wrapped row offsets: next state row, index row two ahead, output rows
    size_t o_in, o_idx, o_now, o_out;

    __device__ __forceinline__ size_t next_row(size_t o) const {
        o += pitch;
        return o == size_t(ny) * pitch ? 0 : o;
    }

    template <int B>
    __device__ __forceinline__ void fetch_state(size_t ro) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int p = plane_of<P>(c);
            if (p >= 0) vload<T, LX>(in + p * plane + ro, qbuf[B][c]);
        }
    }

    template <int B>
    __device__ __forceinline__ void lookup_next() {
#pragma unroll
        for (int x = 0; x < LX; ++x) {
            const MedRec<T> *r = table + ibuf[B][x];
            knext[x] = r->c;
            if constexpr (VIN) vnext[x] = r->v;
        }
    }

    // One march iteration for input row J; PH = (J - J0) mod 4 picks the
    // ring slots, its parity the prefetch buffers.  On entry qbuf[B] holds row
    // J, knext/vnext its records, ibuf[B^1] the indices of row J+1.
    template <int PH>
    __device__ __forceinline__ void iter(int J, int xl, int y_lo, int y_hi, int lane) {
        constexpr int S0 = PH, S1 = (PH + 3) & 3, S2 = (PH + 2) & 3, S3 = (PH + 1) & 3;
        constexpr int B = PH & 1;
        T (&q)[6][LX] = qbuf[B];
        CV kv[LX];
#pragma unroll
        for (int x = 0; x < LX; ++x) {
            kring[S0][x] = knext[x];
            if constexpr (VIN) kv[x] = vnext[x];
        }
        // loads for later rows fly while this row computes: the next row's
        // state, the indices two rows ahead, the next row's records
        fetch_state<B ^ 1>(o_in + xl);
        o_in = next_row(o_in);
        iload<T, LX>(midx + o_idx + xl, ibuf[B]);
        o_idx = next_row(o_idx);
        lookup_next<B ^ 1>();

        // the previous step's V_x, V_y on the entering row
        if constexpr (VIN) {
#pragma unroll
            for (int x = 0; x < LX; ++x) {
                T s[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) s[c] = plane_of<P>(c) >= 0 ? q[c][x] : T(0);
                apply_potential<T, P, VM>(s, kv[x]);
#pragma unroll
                for (int c = 0; c < 6; ++c)
                    if (plane_of<P>(c) >= 0) q[c][x] = s[c];
            }
        }
        apply_ux<T, P, LX>(q, kring[S0]);                          // U_x, row J

        // lanes whose columns are all inside [4, W - 4) hold output columns
        const bool lane_out = lane * LX >= 4 && lane * LX + LX <= W - 4;
        // planes U_y does not touch are final for row J now
        if (J >= y_lo && J < y_hi && lane_out) {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const int p = plane_of<P>(c);
                if (p >= 0 && !in_y_pair<P>(c)) vstore<T, LX>(out + p * plane + o_now + xl, q[c]);
            }
        }
        o_now = next_row(o_now);

        uy_local<T, P, LX, 0>(q, kring[S0]);                       // L1, row J
        uy_neighbour<T, P, LX, 1>(q, carry[0], kring[S0]);         // L2 -> row J-1
        uy_local<T, P, LX, 2>(q, kring[S1]);                       // L3, row J-1
        uy_neighbour<T, P, LX, 3>(q, carry[1], kring[S2]);         // L4 -> row J-2
        uy_local<T, P, LX, 4>(q, kring[S2]);                       // L5, row J-2
        uy_neighbour<T, P, LX, 5>(q, carry[2], kring[S3]);         // L6 -> row J-3
        uy_local<T, P, LX, 6>(q, kring[S3]);                       // L7, row J-3
        uy_neighbour<T, P, LX, 7>(q, carry[3], kring[S3]);         // L8 -> row J-4

        // the U_y planes of row J - 4 are final
        const int R = J - LAG;
        if (R >= y_lo && R < y_hi && lane_out) {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const int p = plane_of<P>(c);
                if (p >= 0 && in_y_pair<P>(c)) vstore<T, LX>(out + p * plane + o_out + xl, q[c]);
            }
        }
        o_out = next_row(o_out);
    }

    __device__ __forceinline__ void run() {
        const int lane = threadIdx.x & 31;
        const int item = blockIdx.x * WARPS + (threadIdx.x >> 5);
        if (item >= n_items) return;
        const int wx = item % n_wx, wy = item / n_wx;
        // window columns [x0, x0 + W), x0 = wx*WOUT - 4 (periodic)
        int xl = wx * WOUT - 4 + lane * LX;
        const bool lane_store_ok = xl >= 0 ? xl < nx : true;
        xl %= nx;
        if (xl < 0) xl += nx;
        const int y_lo = wy * seg_h;
        const int y_hi = min(ny, y_lo + seg_h);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c)
#pragma unroll
                    for (int x = 0; x < LX; ++x) carry[a][b][c][x] = T(0);
        // rows y_lo-4 .. y_hi+3 enter; rows y_lo .. y_hi-1 are stored
        const int J0 = y_lo - LAG;
        const int J1 = y_hi + LAG;  // exclusive
        // lanes whose output columns fall beyond nx (last window) must not
        // store: make their segment empty
        const int st_lo = lane_store_ok ? y_lo : y_hi;
        const size_t o0 = size_t(wrap(J0, ny)) * pitch;
        fetch_state<0>(o0 + xl);
        iload<T, LX>(midx + o0 + xl, ibuf[0]);
        o_in = next_row(o0);
        iload<T, LX>(midx + o_in + xl, ibuf[1]);
        o_idx = next_row(o_in);
        o_now = o0;
        o_out = size_t(wrap(J0 - LAG, ny)) * pitch;
        lookup_next<0>();
        for (int J = J0; J < J1; J += 4) {
            iter<0>(J + 0, xl, st_lo, y_hi, lane);
            iter<1>(J + 1, xl, st_lo, y_hi, lane);
            iter<2>(J + 2, xl, st_lo, y_hi, lane);
            iter<3>(J + 3, xl, st_lo, y_hi, lane);
        }
    }
};

// Blocks per SM the register allocation must allow: the FP32 two-column
// E_z variant is held to 128 registers (16 warps per SM); the others take
// what they need.
template <typename T, int P, int LX> constexpr int min_blocks() {
    return (sizeof(T) == 4 && P == 3 && LX == 2) ? 4 : 1;
}

template <typename T, int P, int LX, int VM, bool VIN>
__global__ void __launch_bounds__(32 * WARPS, min_blocks<T, P, LX>())
k_step_march(const T *__restrict__ in, T *__restrict__ out, const uint32_t *__restrict__ midx,
             const MedRec<T> *__restrict__ table, int nx, int ny, int pitch, size_t plane,
             int seg_h, int n_wx, int n_items) {
    March<T, P, LX, VM, VIN> m;
    m.in = in;
    m.out = out;
    m.midx = midx;
    m.table = table;
    m.nx = nx;
    m.ny = ny;
    m.pitch = pitch;
    m.plane = plane;
    m.seg_h = seg_h;
    m.n_wx = n_wx;
    m.n_items = n_items;
    m.run();
}

// Segment height: as many equal work items as resident warp slots (one full
// wave, or several if a segment would exceed 512 rows), each at least 32 rows
// and a multiple of 4.
inline int pick_segment(int ny, int n_wx, long long resident_warps) {
    if (resident_warps < 1) resident_warps = 1;
    long long waves = 1;
    while ((long long)n_wx * ny / (resident_warps * waves) > 512) ++waves;
    long long n_wy = resident_warps * waves / n_wx;
    if (n_wy < 1) n_wy = 1;
    int seg = int((ny + n_wy - 1) / n_wy);
    if (seg < 32) seg = 32;
    return (seg + 3) / 4 * 4;
}

template <typename T, int P, int LX, int VM, bool VIN>
cudaError_t launch_t(qla_ctx *c, const void *in, void *out) {
    constexpr int WOUT = 32 * LX - 8;
    auto kern = k_step_march<T, P, LX, VM, VIN>;
    static int blocks_per_sm = -1;  // per instantiation, per process
    if (blocks_per_sm < 0) {
        int b = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 32 * WARPS, 0);
        if (e != cudaSuccess) return e;
        blocks_per_sm = b > 0 ? b : 1;
    }
    const int n_wx = (c->nx + WOUT - 1) / WOUT;
    int seg = c->march_seg;
    if (seg <= 0)
        seg = pick_segment(c->ny, n_wx, (long long)blocks_per_sm * WARPS * c->num_sms);
    else
        seg = (seg + 3) / 4 * 4;
    const int n_wy = (c->ny + seg - 1) / seg;
    const int n_items = n_wx * n_wy;
    const int blocks = (n_items + WARPS - 1) / WARPS;
    kern<<<blocks, 32 * WARPS, 0, c->stream>>>(
        static_cast<const T *>(in), static_cast<T *>(out), c->midx,
        static_cast<const MedRec<T> *>(c->table), c->nx, c->ny, c->pitch, c->plane_elems, seg,
        n_wx, n_items);
    return cudaGetLastError();
}

// The previous step's potential operator is applied to each entering row
// when one is pending (see qla_ctx::pending_v).
template <typename T, int P, int LX>
cudaError_t launch_vm(qla_ctx *c, const void *in, void *out, bool vin) {
    switch (c->vmode) {
    case V_ROTATION:
        return vin ? launch_t<T, P, LX, V_ROTATION, true>(c, in, out)
                   : launch_t<T, P, LX, V_ROTATION, false>(c, in, out);
    case V_LITERAL:
        return vin ? launch_t<T, P, LX, V_LITERAL, true>(c, in, out)
                   : launch_t<T, P, LX, V_LITERAL, false>(c, in, out);
    default: return launch_t<T, P, LX, V_NONE, false>(c, in, out);
    }
}

}  // namespace

// Columns per lane: 2 or 4 for FP32 E_z contexts (tunable, default 2: at
// 128 registers four warps per scheduler stay resident, which outweighs the
// wider window's smaller halo), 2 otherwise.
int march_lane_cols(const qla_ctx *c) {
    if (c->prec == QLA_FP32 && c->P == 3) return c->march_lx == 4 ? 4 : 2;
    return 2;
}

bool march_supported(const qla_ctx *c) {
    const int lx = march_lane_cols(c);
    return c->nx % lx == 0 && c->nx >= 32 * lx && c->ny >= 8;
}

cudaError_t launch_step_march(qla_ctx *c, const void *in, void *out, bool vin) {
    if (c->prec == QLA_FP64)
        return c->P == 6 ? launch_vm<double, 6, 2>(c, in, out, vin)
                         : launch_vm<double, 3, 2>(c, in, out, vin);
    if (c->P == 6) return launch_vm<float, 6, 2>(c, in, out, vin);
    return march_lane_cols(c) == 2 ? launch_vm<float, 3, 2>(c, in, out, vin)
                                   : launch_vm<float, 3, 4>(c, in, out, vin);
}

}  // namespace qla
