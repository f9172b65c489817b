// Device-side machinery of the marching QLA step (see qla_step_march.cu for
// the algorithm): bond-layer rotations for U_x with warp shuffles, the U_y
// row pipeline, row staging through shared memory, and the per-warp work
// item.  Included by the single-lattice and the batched kernels.
#pragma once

#include "qla_internal.h"

namespace qla {
namespace march {


constexpr int WARPS = 4;           // independent warps per CTA
constexpr int LAG = 4;             // rows between U_y input and output

template <typename T, int LX> struct Vec;
template <> struct Vec<float, 4> { using type = float4; };
template <> struct Vec<float, 2> { using type = float2; };
template <> struct Vec<double, 2> { using type = double2; };
template <> struct Vec<dsf, 2> { using type = float4; };   // two (hi, lo) pairs

// Streamed data (state planes, index rows) is read through L2 only, so that
// L1 keeps the medium records, which every row looks up.
template <typename T, int LX>
__device__ __forceinline__ void vload(const T *p, T (&v)[LX]) {
    const auto t = __ldcg(reinterpret_cast<const typename Vec<T, LX>::type *>(p));
    if constexpr (std::is_same<T, dsf>::value) { v[0] = dsf(t.x, t.y); v[1] = dsf(t.z, t.w); }
    else if constexpr (LX == 4) { v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
    else { v[0] = t.x; v[1] = t.y; }
}

template <typename T, int LX>
__device__ __forceinline__ void vstore(T *p, const T (&v)[LX]) {
    typename Vec<T, LX>::type t;
    if constexpr (std::is_same<T, dsf>::value) { t = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo); }
    else if constexpr (LX == 4) { t.x = v[0]; t.y = v[1]; t.z = v[2]; t.w = v[3]; }
    else { t.x = v[0]; t.y = v[1]; }
    *reinterpret_cast<typename Vec<T, LX>::type *>(p) = t;
}

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_dn1(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ dsf shfl_up1(dsf v) { return dsf(shfl_up1(v.hi), shfl_up1(v.lo)); }
__device__ __forceinline__ dsf shfl_dn1(dsf v) { return dsf(shfl_dn1(v.hi), shfl_dn1(v.lo)); }

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

// Per-lane asynchronous global -> shared copies (no registers held while
// the data is in flight); each lane later reads back only what it copied.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gmem), "n"(BYTES)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

constexpr int NSLOT = 4;   // rows staged per warp: the current one and 3 ahead

// UNI: a work item whose every entering site shares one record (a plateau
// of the medium, where the four neighbours of each site carry its n): the
// collision coefficients are one warp-uniform value `ku` instead of the
// register ring (no index rows staged, no record lookups, and no potential
// step: V is the identity on shared-record sites).  Given the coefficients
// from the constant bank, the rotations read one register operand fewer.
template <typename T, int P, int LX, int VM, bool VIN, bool UNI = false>
struct March {
    using CC = typename Coef<T>::C;
    using CV = typename Coef<T>::V;
    static constexpr int W = 32 * LX;   // window columns
    static constexpr int WOUT = W - 8;  // stored columns
    // one staged row: the set's planes of W values, then W record indices
    struct Slot {
        T q[nplanes<P>()][W];
        uint32_t idx[W];
    };

    // this lane's column in each array (offsets below are element offsets
    // of a row start, 32-bit: ny * pitch < 2^31 is checked on the host)
    const T *in;
    T *out;
    const uint32_t *midx;
    const MedRec<T> *table;
    uint32_t plane, total;  // plane stride; ny * pitch
    int pitch;
    Slot *ring;             // this warp's NSLOT staged rows
    int lc;                 // this lane's first column in the window

    // state carried along the march
    T carry[4][2][2][LX];   // [neighbour layer][pair][value][x]
    CC kring[LAG][LX];      // collision coefficients of the rows in flight
    CV vnext[LX];           // row J+1's potential coefficients
    // whether row J+1's site has its own record: shared records (index below
    // UNIFORM_SLOTS) belong to sites whose four neighbours carry their n, so
    // beta = 0 and V is exactly the identity there (cos 1, sin 0 in FP64;
    // 1 - cos 0, sin 0 in FP32): skipping it changes no bit
    bool vlive[LX];
    // FP64 looks row J+1's records up early (their latency hides behind the
    // row's arithmetic) and copies them into the ring at the next row; FP32
    // and double-single load them straight into the ring slot that frees at
    // the end of the row, which saves the copies (measured: FP32 faster,
    // FP64 slower the other way round)
    static constexpr bool EARLY = std::is_same<T, double>::value;
    CC knext[EARLY ? LX : 1];
    CC ku[UNI ? LX : 1];    // UNI: the item's coefficients, copies of one value
    __device__ __forceinline__ void set_uniform(CC k) {
#pragma unroll
        for (int x = 0; x < (UNI ? LX : 1); ++x) ku[x] = k;
    }
    // coefficients of the row in ring slot S
    template <int S>
    __device__ __forceinline__ const CC (&ring_coef() const)[LX] {
        if constexpr (UNI) return ku;
        else return kring[S];
    }
    // row offsets: next row to stage, the two output rows
    uint32_t o_in, o_now, o_out;

    __device__ __forceinline__ uint32_t next_row(uint32_t o) const {
        o += uint32_t(pitch);
        return o == total ? 0u : o;
    }

    // Stage the row at offset o_in into slot `sl` (one commit group).
    __device__ __forceinline__ void stage_into(Slot &sl) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int p = plane_of<P>(c);
            if (p >= 0)
                cp_async<LX * sizeof(T)>(&sl.q[slot_of<P>(c)][lc], in + p * plane + o_in);
        }
        if constexpr (!UNI) cp_async<LX * 4>(&sl.idx[lc], midx + o_in);
        cp_async_commit();
        o_in = next_row(o_in);
    }
    template <int S>
    __device__ __forceinline__ void stage() { stage_into(ring[S]); }

    // Row J + 1's records (staging slot S) into ring slot K of the collision
    // coefficients and into vnext.
    template <int S, int K>
    __device__ __forceinline__ void lookup_next() {
#pragma unroll
        for (int x = 0; x < LX; ++x) {
            const uint32_t id = ring[S].idx[lc + x];
            const MedRec<T> *r = table + id;
            if constexpr (EARLY) knext[x] = r->c;
            else kring[K][x] = r->c;
            if constexpr (VIN) {
                vlive[x] = id >= uint32_t(UNIFORM_SLOTS);
                if (vlive[x]) vnext[x] = r->v;
            }
        }
    }

    // One march iteration for input row J; PH = (J - J0) mod 4 picks the
    // register ring slots and the staging slot of row J.  On entry kring[PH]
    // (FP64: knext) and vnext hold row J's records.  Rows J and J - 4 are stored when they
    // fall in [st_lo, st_lo + st_n).
    template <int PH>
    __device__ __forceinline__ void iter(int J, int st_lo, unsigned st_n) {
        iter_body<PH>(J, st_lo, st_n, ring[PH], ring[(PH + 3) & (NSLOT - 1)]);
    }
    // UNI: the same with the staging slots chosen at run time (phase ph of
    // row J), so that the march loop need not be unrolled four times: the
    // four-column body is large, and four copies of it overflowed the
    // instruction cache (no-instruction stalls 1.49 per issue)
    __device__ __forceinline__ void iter_rt(int J, int st_lo, unsigned st_n, int ph) {
        static_assert(UNI, "only plateau items have no ring slots to name");
        iter_body<0>(J, st_lo, st_n, ring[ph], ring[(ph + 3) & (NSLOT - 1)]);
    }
    // cur: row J's staging slot; nxt: the slot row J - 1 used, refilled with
    // row J + 3
    template <int PH>
    __device__ __forceinline__ void iter_body(int J, int st_lo, unsigned st_n, Slot &cur,
                                              Slot &nxt) {
        constexpr int S0 = PH, S1 = (PH + 3) & 3, S2 = (PH + 2) & 3, S3 = (PH + 1) & 3;
        // stage row J + 3 into the slot row J - 1 used; wait for row J + 1
        stage_into(nxt);
        cp_async_wait<NSLOT - 2>();
        T q[6][LX];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (plane_of<P>(c) >= 0) {
#pragma unroll
                for (int x = 0; x < LX; ++x) q[c][x] = cur.q[slot_of<P>(c)][lc + x];
            }
        }
        if constexpr (EARLY && !UNI) {
#pragma unroll
            for (int x = 0; x < LX; ++x) kring[S0][x] = knext[x];
        }
        // the previous step's V_x, V_y on the entering row
        if constexpr (VIN && !UNI) {
#pragma unroll
            for (int x = 0; x < LX; ++x) {
                if (!vlive[x]) continue;
                T s[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) s[c] = plane_of<P>(c) >= 0 ? q[c][x] : T(0);
                apply_potential<T, P, VM>(s, vnext[x]);
#pragma unroll
                for (int c = 0; c < 6; ++c)
                    if (plane_of<P>(c) >= 0) q[c][x] = s[c];
            }
        }
        // (FP64) row J + 1's records fly while this row computes
        if constexpr (EARLY && !UNI) lookup_next<(PH + 1) & (NSLOT - 1), S3>();

        apply_ux<T, P, LX>(q, ring_coef<S0>());                    // U_x, row J

        // planes U_y does not touch are final for row J now
        if (unsigned(J - st_lo) < st_n) {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const int p = plane_of<P>(c);
                if (p >= 0 && !in_y_pair<P>(c)) vstore<T, LX>(out + p * plane + o_now, q[c]);
            }
        }
        o_now = next_row(o_now);

        uy_local<T, P, LX, 0>(q, ring_coef<S0>());                 // L1, row J
        uy_neighbour<T, P, LX, 1>(q, carry[0], ring_coef<S0>());   // L2 -> row J-1
        uy_local<T, P, LX, 2>(q, ring_coef<S1>());                 // L3, row J-1
        uy_neighbour<T, P, LX, 3>(q, carry[1], ring_coef<S2>());   // L4 -> row J-2
        uy_local<T, P, LX, 4>(q, ring_coef<S2>());                 // L5, row J-2
        uy_neighbour<T, P, LX, 5>(q, carry[2], ring_coef<S3>());   // L6 -> row J-3
        uy_local<T, P, LX, 6>(q, ring_coef<S3>());                 // L7, row J-3
        uy_neighbour<T, P, LX, 7>(q, carry[3], ring_coef<S3>());   // L8 -> row J-4
        // row J - 3's coefficients (slot S3) are dead: row J + 1's records
        // go straight into that slot
        if constexpr (!EARLY && !UNI) lookup_next<(PH + 1) & (NSLOT - 1), S3>();

        // the U_y planes of row J - 4 are final
        if (unsigned(J - LAG - st_lo) < st_n) {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const int p = plane_of<P>(c);
                if (p >= 0 && in_y_pair<P>(c)) vstore<T, LX>(out + p * plane + o_out, q[c]);
            }
        }
        o_out = next_row(o_out);
    }

    // Process work item `item` (window item % n_wx, row segment item / n_wx)
    // of the lattice whose arrays are in/out/midx/table; warp_ring is this
    // warp's staging buffer.
    __device__ __forceinline__ void run_item(int nx, int ny, int seg_h, int n_wx, int item,
                                             Slot *warp_ring) {
        const int wx = item % n_wx, wy = item / n_wx;
        const int x_out = wx * WOUT;
        run_unit(nx, ny, x_out, min(WOUT, nx - x_out), wy * seg_h, min(ny, wy * seg_h + seg_h),
                 warp_ring);
    }

    // The same for an explicit unit: store columns [x_out, x_out + w_out)
    // (w_out <= WOUT, x_out + w_out <= nx, both multiples of LX) of rows
    // [y_lo, y_hi); the window starts 4 columns left of x_out (periodic).
    __device__ __forceinline__ void run_unit(int nx, int ny, int x_out, int w_out, int y_lo,
                                             int y_hi, Slot *warp_ring) {
        const int lane = threadIdx.x & 31;
        ring = warp_ring;
        lc = lane * LX;
        // window columns [x0, x0 + W), x0 = x_out - 4 (periodic)
        int xl = x_out - 4 + lane * LX;
        xl %= nx;
        if (xl < 0) xl += nx;
        in += xl;
        out += xl;
        midx += xl;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c)
#pragma unroll
                    for (int x = 0; x < LX; ++x) carry[a][b][c][x] = T(0);
        // the coefficient slots of the rows before J0 are read by the first
        // iterations (their results reach halo rows only); they must hold
        // defined values, or the compiler may substitute any register
#pragma unroll
        for (int a = 0; a < LAG; ++a)
#pragma unroll
            for (int x = 0; x < LX; ++x) kring[a][x] = CC{};
        // rows y_lo-4 .. y_hi+3 enter; rows y_lo .. y_hi-1 are stored by the
        // lanes whose columns are all inside [4, 4 + w_out)
        const int J0 = y_lo - LAG;
        const int J1 = y_hi + LAG;  // exclusive
        const bool lane_out = lc >= 4 && lc + LX <= 4 + w_out;
        const unsigned st_n = lane_out ? unsigned(y_hi - y_lo) : 0u;
        o_in = uint32_t(wrap(J0, ny)) * uint32_t(pitch);
        o_now = o_in;
        o_out = uint32_t(wrap(J0 - LAG, ny)) * uint32_t(pitch);
        // rows J0, J0+1, J0+2 in flight; row J0's records before the loop
        stage<0>();
        stage<1>();
        stage<2>();
        cp_async_wait<2>();
        if constexpr (UNI && LX == 4) {
            // two rows per loop body (all-plateau 16384^2 lattice, 256-row
            // segments: 1.43 ms per step against 1.50 ms with one row and
            // 1.47 ms with four rows on compile-time slots)
#pragma unroll 2
            for (int J = J0; J < J1; ++J) iter_rt(J, y_lo, st_n, (J - J0) & (NSLOT - 1));
        } else {
            if constexpr (!UNI) lookup_next<0, 0>();
            for (int J = J0; J < J1; J += 4) {
                iter<0>(J + 0, y_lo, st_n);
                iter<1>(J + 1, y_lo, st_n);
                iter<2>(J + 2, y_lo, st_n);
                iter<3>(J + 3, y_lo, st_n);
            }
        }
        cp_async_wait<0>();
    }
};


}  // namespace march
}  // namespace qla
