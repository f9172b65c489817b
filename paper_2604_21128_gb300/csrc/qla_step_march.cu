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
//  * V_x, V_y (Eqs. 2e11-2e13) act on that row, which is then stored.
// Amplitudes untouched by U_y wait in a four-row register ring.  The
// collision coefficients of the four rows in flight also sit in a ring.  The
// march loop is unrolled by four so that every ring slot is a fixed register.
#include "qla_internal.h"

namespace qla {
namespace {

constexpr int WARPS = 4;           // independent warps per CTA
constexpr int LAG = 4;             // rows between U_y input and output

template <typename T, int LX> struct Vec;
template <> struct Vec<float, 4> { using type = float4; };
template <> struct Vec<float, 2> { using type = float2; };
template <> struct Vec<double, 2> { using type = double2; };

template <typename T, int LX>
__device__ __forceinline__ void vload(const T *p, T (&v)[LX]) {
    const auto t = *reinterpret_cast<const typename Vec<T, LX>::type *>(p);
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
template <typename T, int P, int LX, int VM>
struct March {
    using CC = typename Coef<T>::C;
    using CV = typename Coef<T>::V;
    static constexpr int W = 32 * LX;   // window columns
    static constexpr int WOUT = W - 8;  // stored columns

    const T *in;
    T *out;
    const CC *cC;
    const CV *cV;
    int nx, ny, pitch, seg_h, n_wx, n_items;
    size_t plane;

    // state carried along the march
    T carry[4][2][2][LX];   // [neighbour layer][pair][value][x]
    T delay[LAG][6][LX];    // planes not in a U_y pair, by row phase
    CC kring[LAG][LX];      // collision coefficients of the rows in flight

    __device__ __forceinline__ size_t row_off(int r) const {
        r %= ny;
        if (r < 0) r += ny;
        return size_t(r) * pitch;
    }

    // One march iteration for input row J; PH = J mod 4 (ring slot of J).
    template <int PH>
    __device__ __forceinline__ void iter(int J, int xl, int y_lo, int y_hi, int lane) {
        constexpr int S0 = PH, S1 = (PH + 3) & 3, S2 = (PH + 2) & 3, S3 = (PH + 1) & 3;
        const size_t ro = row_off(J) + xl;
        T q[6][LX];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int p = plane_of<P>(c);
            if (p >= 0) vload<T, LX>(in + p * plane + ro, q[c]);
        }
#pragma unroll
        for (int x = 0; x < LX; ++x) kring[S0][x] = cC[ro + x];
        // coefficients of V for the row leaving the pipeline (J - 4)
        const int R = J - LAG;
        const size_t ro_out = row_off(R) + xl;
        CV kv[LX];
#pragma unroll
        for (int x = 0; x < LX; ++x) kv[x] = cV[ro_out + x];

        apply_ux<T, P, LX>(q, kring[S0]);                          // U_x, row J
        uy_local<T, P, LX, 0>(q, kring[S0]);                       // L1, row J
        uy_neighbour<T, P, LX, 1>(q, carry[0], kring[S0]);         // L2 -> row J-1
        uy_local<T, P, LX, 2>(q, kring[S1]);                       // L3, row J-1
        uy_neighbour<T, P, LX, 3>(q, carry[1], kring[S2]);         // L4 -> row J-2
        uy_local<T, P, LX, 4>(q, kring[S2]);                       // L5, row J-2
        uy_neighbour<T, P, LX, 5>(q, carry[2], kring[S3]);         // L6 -> row J-3
        uy_local<T, P, LX, 6>(q, kring[S3]);                       // L7, row J-3
        uy_neighbour<T, P, LX, 7>(q, carry[3], kring[S3]);         // L8 -> row J-4

        // planes untouched by U_y: swap the row J values into the ring slot
        // that held row J-4's
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (plane_of<P>(c) < 0 || in_y_pair<P>(c)) continue;
#pragma unroll
            for (int x = 0; x < LX; ++x) {
                const T t = delay[S0][c][x];
                delay[S0][c][x] = q[c][x];
                q[c][x] = t;
            }
        }
        if constexpr (VM != V_NONE) {
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
        // store row R if it is in this segment and the lane holds output
        // columns (lanes whose columns are all inside [4, W - 4))
        const bool lane_out = lane * LX >= 4 && lane * LX + LX <= W - 4;
        if (R >= y_lo && R < y_hi && lane_out) {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const int p = plane_of<P>(c);
                if (p >= 0) vstore<T, LX>(out + p * plane + ro_out, q[c]);
            }
        }
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
#pragma unroll
        for (int a = 0; a < LAG; ++a)
#pragma unroll
            for (int c = 0; c < 6; ++c)
#pragma unroll
                for (int x = 0; x < LX; ++x) delay[a][c][x] = T(0);
        // rows y_lo-4 .. y_hi+3 enter; rows y_lo .. y_hi-1 leave and are stored
        const int J0 = y_lo - LAG;
        const int J1 = y_hi + LAG;  // exclusive
        // lanes whose output columns fall beyond nx (last window) must not
        // store: make their segment empty
        const int st_lo = lane_store_ok ? y_lo : y_hi;
        for (int J = J0; J < J1; J += 4) {
            iter<0>(J + 0, xl, st_lo, y_hi, lane);
            iter<1>(J + 1, xl, st_lo, y_hi, lane);
            iter<2>(J + 2, xl, st_lo, y_hi, lane);
            iter<3>(J + 3, xl, st_lo, y_hi, lane);
        }
    }
};

template <typename T, int P, int LX, int VM>
__global__ void __launch_bounds__(32 * WARPS)
k_step_march(const T *__restrict__ in, T *__restrict__ out,
             const typename Coef<T>::C *__restrict__ cC,
             const typename Coef<T>::V *__restrict__ cV, int nx, int ny, int pitch,
             size_t plane, int seg_h, int n_wx, int n_items) {
    March<T, P, LX, VM> m;
    m.in = in;
    m.out = out;
    m.cC = cC;
    m.cV = cV;
    m.nx = nx;
    m.ny = ny;
    m.pitch = pitch;
    m.plane = plane;
    m.seg_h = seg_h;
    m.n_wx = n_wx;
    m.n_items = n_items;
    m.run();
}

template <typename T, int P> constexpr int lanes_cols() {
    return (sizeof(T) == 4 && P == 3) ? 4 : 2;
}

template <typename T, int P, int VM>
cudaError_t launch_t(qla_ctx *c, const void *in, void *out) {
    constexpr int LX = lanes_cols<T, P>();
    constexpr int WOUT = 32 * LX - 8;
    const int n_wx = (c->nx + WOUT - 1) / WOUT;
    // segment height: about four work items per resident warp slot, rows a
    // multiple of 4, at least 64
    const long long want_items = 4LL * c->num_sms * 12;
    int seg = int((long long)c->ny * n_wx / (want_items > 0 ? want_items : 1));
    seg = seg < 64 ? 64 : seg;
    seg = (seg + 3) / 4 * 4;
    if (seg > c->ny) seg = (c->ny + 3) / 4 * 4;
    const int n_wy = (c->ny + seg - 1) / seg;
    const int n_items = n_wx * n_wy;
    const int blocks = (n_items + WARPS - 1) / WARPS;
    k_step_march<T, P, LX, VM><<<blocks, 32 * WARPS, 0, c->stream>>>(
        static_cast<const T *>(in), static_cast<T *>(out),
        static_cast<const typename Coef<T>::C *>(c->coefC),
        static_cast<const typename Coef<T>::V *>(c->coefV), c->nx, c->ny, c->pitch,
        c->plane_elems, seg, n_wx, n_items);
    return cudaGetLastError();
}

template <typename T, int P>
cudaError_t launch_vm(qla_ctx *c, const void *in, void *out) {
    switch (c->vmode) {
    case V_ROTATION: return launch_t<T, P, V_ROTATION>(c, in, out);
    case V_LITERAL:  return launch_t<T, P, V_LITERAL>(c, in, out);
    default:         return launch_t<T, P, V_NONE>(c, in, out);
    }
}

}  // namespace

bool march_supported(const qla_ctx *c) {
    const int lx = (c->prec == QLA_FP32 && c->P == 3) ? 4 : 2;
    return c->nx % lx == 0 && c->nx >= 32 * lx && c->ny >= 8;
}

cudaError_t launch_step_march(qla_ctx *c, const void *in, void *out) {
    if (c->prec == QLA_FP64)
        return c->P == 6 ? launch_vm<double, 6>(c, in, out) : launch_vm<double, 3>(c, in, out);
    return c->P == 6 ? launch_vm<float, 6>(c, in, out) : launch_vm<float, 3>(c, in, out);
}

}  // namespace qla
