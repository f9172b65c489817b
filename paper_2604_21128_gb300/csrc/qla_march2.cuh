// Packed-pair variant of the marching QLA step for FP32 E_z contexts.
//
// The step is the one of qla_march.cuh (bond layers for U_x, a register
// pipeline along y for U_y, the pending potential step on entering rows),
// with another assignment of columns to lanes: in a 64-column window lane l
// holds columns l and l + 32 as the two halves of a float2, and every
// rotation acts on both at once with packed FP32x2 arithmetic (fma.rn.f32x2,
// mul.rn.f32x2).  The operations per element and their order are those of
// the scalar rotate(), so results are bitwise those of the other kernels;
// the packed form issues half the arithmetic instructions.
//
// Why columns 32 apart: a bond layer of U_x pairs a column with its left or
// right neighbour, and with this layout the neighbours of both halves live
// in the same neighbouring lane (lane l - 1 or l + 1) in the same half,
// except at the seam between the halves (lane 0's high column needs lane
// 31's low one, and back).  Each bond layer therefore costs four shuffles
// and two selects, and no register ever has to be re-paired.
//
// Rows are staged into the warp's shared-memory ring by 16-byte cp.async
// chunks (two per lane per row: three planes and the index row, 16 chunks
// each), so a lane reads columns another lane copied: a __syncwarp() after
// the wait publishes them, and one before the next copy keeps it from
// overwriting a row still being read.
#pragma once

#include "qla_march.cuh"

namespace qla {
namespace march {

// Pair arithmetic: float2 values and the packed intrinsics (one rounding
// per fma.rn / mul.rn on each half; negation of an operand is folded into
// the instruction).
struct PairF2 {
    using T = float2;
    __device__ static __forceinline__ T make(float lo, float hi) { return make_float2(lo, hi); }
    __device__ static __forceinline__ float lo(T v) { return v.x; }
    __device__ static __forceinline__ float hi(T v) { return v.y; }
    __device__ static __forceinline__ T fma(T a, T b, T c) { return __ffma2_rn(a, b, c); }
    __device__ static __forceinline__ T mul(T a, T b) { return __fmul2_rn(a, b); }
    __device__ static __forceinline__ T neg(T a) { return make_float2(-a.x, -a.y); }
};

// Two-word collision coefficients of two columns: (c_hi, s_hi, c_lo, s_lo)
// of Coef<float>, one column per half.
template <typename PO> struct K2 {
    typename PO::T ch, sh, cl, sl;
    __device__ __forceinline__ void copy_from(const K2 &o) {
        ch = o.ch;
        sh = o.sh;
        cl = o.cl;
        sl = o.sl;
    }
};

// (a, b) <- [[c, -G s], [G s, c]] (a, b) on both halves: per element the
// operations of rotate(float &, float &, float4, float) in the same order.
template <typename PO, int G>
__device__ __forceinline__ void rotate2(typename PO::T &a, typename PO::T &b, const K2<PO> &k) {
    using T = typename PO::T;
    // G s and -G s, high and low words
    const T shp = G > 0 ? k.sh : PO::neg(k.sh), slp = G > 0 ? k.sl : PO::neg(k.sl);
    const T shn = PO::neg(shp), sln = PO::neg(slp);
    const T na = PO::fma(k.ch, a, PO::fma(shn, b, PO::fma(k.cl, a, PO::mul(sln, b))));
    const T nb = PO::fma(k.ch, b, PO::fma(shp, a, PO::fma(k.cl, b, PO::mul(slp, a))));
    a = na;
    b = nb;
}

// mask ? a : b for a mask of all ones or all zeros, as one bit operation:
// the seam selects of the bond layers take no predicate register (several
// predicates live across the whole march otherwise crowd the predicate file).
__device__ __forceinline__ float bitsel(uint32_t mask, float a, float b) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0xE4;"
        : "=r"(d)
        : "r"(__float_as_uint(a)), "r"(__float_as_uint(b)), "r"(mask));
    return __uint_as_float(d);
}

template <typename PO, int G>
__device__ __forceinline__ void bond_rot2(typename PO::T &u, typename PO::T &m, const K2<PO> &k,
                                          bool a_moved) {
    if (a_moved) rotate2<PO, G>(m, u, k);
    else rotate2<PO, G>(u, m, k);
}

// UNI: a plateau item (see March in qla_march.cuh): one coefficient set
// `ku` for every row and column, no index rows, no lookups, no potential
// step.  Not combined with ILV.
template <int VM, bool VIN, typename PO = PairF2, bool ILV = false, bool UNI = false>
struct March2 {
    static_assert(!(ILV && UNI), "the interleaved march has no plateau form");
    using T2 = typename PO::T;
    static constexpr int W = 64;        // window columns (lane l: l and l + 32)
    static constexpr int WOUT = W - 8;  // stored columns
    // one staged row: planes q2, q3, q4 of the window, then its record indices
    struct Slot {
        float q[3][W];
        uint32_t idx[W];
    };

    const float *in;
    float *out;
    const uint32_t *midx;
    const MedRec<float> *table;
    uint32_t plane, total;   // plane stride; ny * pitch
    int pitch;
    Slot *ring;
    int lane, prev, next;    // this lane, the lanes before and after it (mod 32)
    uint32_t first, last;    // all ones on lane 0 / lane 31, else zero
    // the lane's two staging copies: global sources at row 0, shared
    // destinations as byte offsets inside a slot
    const char *src0, *src1;
    uint32_t dst0, dst1;
    bool idx_lane;           // the lane's second copy is of the index row

    T2 carry[4][2];          // U_y neighbour layers: [layer][value]
    K2<PO> kring[LAG];       // collision coefficients of the rows in flight
    K2<PO> ku;               // UNI: the item's coefficients on both halves
    template <int S>
    __device__ __forceinline__ const K2<PO> &ring_coef() const {
        if constexpr (UNI) return ku;
        else return kring[S];
    }
    __device__ __forceinline__ void set_uniform(float4 k) {
        ku.ch = PO::make(k.x, k.x);
        ku.sh = PO::make(k.y, k.y);
        ku.cl = PO::make(k.z, k.z);
        ku.sl = PO::make(k.w, k.w);
    }
    float4 vlo, vhi;         // row J+1's potential coefficients (low, high column)
    // row J+1's sites have their own records (0 or 1; integers, like the
    // other per-lane flags, so that no predicate stays live across the march)
    uint32_t vlive_lo, vlive_hi;
    uint32_t o_in, o_now, o_out;
    // interleaved march (ILV): row J + 1's coefficients, and q2, q3 of row J
    // after U_x, carried into the iteration that runs U_y on row J
    K2<PO> knext;
    T2 p2, p3;

    __device__ __forceinline__ uint32_t next_row(uint32_t o) const {
        o += uint32_t(pitch);
        return o == total ? 0u : o;
    }

    template <int S>
    __device__ __forceinline__ void stage() {
        unsigned char *base = reinterpret_cast<unsigned char *>(ring + S);
        cp_async<16>(base + dst0, src0 + 4ull * o_in);
        if (!UNI || !idx_lane) cp_async<16>(base + dst1, src1 + 4ull * o_in);
        cp_async_commit();
        o_in = next_row(o_in);
    }

    // The records of the row in staging slot S into the coefficients kd and
    // the potential coefficients.
    template <int S>
    __device__ __forceinline__ void lookup_into(K2<PO> &kd) {
        const uint32_t il = ring[S].idx[lane], ih = ring[S].idx[lane + 32];
        const MedRec<float> *rl = table + il, *rh = table + ih;
        // one word per load, straight into its pair: a pair holds the same
        // coefficient of two records, and 16-byte loads of whole records
        // would leave the halves in registers that are not a pair (the
        // compiler then rebuilds the pair at every use)
        const float *wl = reinterpret_cast<const float *>(&rl->c);
        const float *wh = reinterpret_cast<const float *>(&rh->c);
        kd.ch = PO::make(__ldg(wl + 0), __ldg(wh + 0));
        kd.sh = PO::make(__ldg(wl + 1), __ldg(wh + 1));
        kd.cl = PO::make(__ldg(wl + 2), __ldg(wh + 2));
        kd.sl = PO::make(__ldg(wl + 3), __ldg(wh + 3));
        if constexpr (VIN) {
            vlive_lo = il >= uint32_t(UNIFORM_SLOTS) ? 1u : 0u;
            vlive_hi = ih >= uint32_t(UNIFORM_SLOTS) ? 1u : 0u;
            if (vlive_lo) vlo = rl->v;
            if (vlive_hi) vhi = rh->v;
        }
    }
    template <int S, int K>
    __device__ __forceinline__ void lookup_next() { lookup_into<S>(kring[K]); }

    // The pending V_x, V_y at one column (the E_z triple).
    __device__ __forceinline__ void potential(float &q2, float &q3, float &q4, float4 kv) {
        float s[6] = {0.0f, 0.0f, q2, q3, q4, 0.0f};
        apply_potential<float, 3, VM>(s, kv);
        q2 = s[2];
        q3 = s[3];
        q4 = s[4];
    }

    // Partner of every column's u in a bond layer: m of the column to the
    // left (shift -1) or to the right (shift +1), and the way back.
    __device__ __forceinline__ T2 take_left(T2 m) const {
        const float ml = PO::lo(m), mh = PO::hi(m);
        return PO::make(__shfl_sync(0xffffffffu, ml, prev),
                        __shfl_sync(0xffffffffu, bitsel(last, ml, mh), prev));
    }
    __device__ __forceinline__ T2 give_right(T2 mm) const {
        const float ml = PO::lo(mm), mh = PO::hi(mm);
        return PO::make(__shfl_sync(0xffffffffu, bitsel(first, mh, ml), next),
                        __shfl_sync(0xffffffffu, mh, next));
    }
    __device__ __forceinline__ T2 take_right(T2 m) const {
        const float ml = PO::lo(m), mh = PO::hi(m);
        return PO::make(__shfl_sync(0xffffffffu, bitsel(first, mh, ml), next),
                        __shfl_sync(0xffffffffu, mh, next));
    }
    __device__ __forceinline__ T2 give_left(T2 mm) const {
        const float ml = PO::lo(mm), mh = PO::hi(mm);
        return PO::make(__shfl_sync(0xffffffffu, ml, prev),
                        __shfl_sync(0xffffffffu, bitsel(last, ml, mh), prev));
    }

    // U_x layer L on the pair (q2, q4) (Eq. 2e3; q4 is the S14 mover).
    template <int L>
    __device__ __forceinline__ void ux_layer(T2 &q2, T2 &q4, const K2<PO> &k) const {
        constexpr Layer ly = layer_of(L);
        constexpr int G = layer_sign<true, L>();
        if constexpr (ly.mover == 0) {
            rotate2<PO, G>(q2, q4, k);
        } else {
            constexpr bool a_moved = ly.mover != 1;   // S25 moves q2, S14 moves q4
            T2 &m = a_moved ? q2 : q4;
            T2 &u = a_moved ? q4 : q2;
            if constexpr (ly.shift < 0) {
                T2 mm = take_left(m);
                bond_rot2<PO, G>(u, mm, k, a_moved);
                m = give_right(mm);
            } else {
                T2 mm = take_right(m);
                bond_rot2<PO, G>(u, mm, k, a_moved);
                m = give_left(mm);
            }
        }
    }

    // U_y layers on the pair (q2, q3) (Eq. 2e8; q3 is the S03 mover).
    template <int L>
    __device__ __forceinline__ void uy_local(T2 &q2, T2 &q3, const K2<PO> &k) const {
        rotate2<PO, layer_sign<false, L>()>(q2, q3, k);
    }

    template <int L>
    __device__ __forceinline__ void uy_neighbour(T2 &q2, T2 &q3, T2 (&c)[2],
                                                 const K2<PO> &k) const {
        constexpr Layer ly = layer_of(L);
        constexpr int G = layer_sign<false, L>();
        constexpr bool a_moved = ly.mover != 1;   // S25 moves q2, S03 moves q3
        T2 &qm = a_moved ? q2 : q3;
        T2 &qu = a_moved ? q3 : q2;
        const T2 u = qu, m = qm;
        if constexpr (ly.shift < 0) {
            // bond at this row r: (u_r, m_{r-1}); c[0] = m_{r-1} before the
            // layer, c[1] = u_{r-1} after it
            T2 uu = u, mm = c[0];
            bond_rot2<PO, G>(uu, mm, k, a_moved);
            qu = c[1];
            qm = mm;
            c[0] = m;
            c[1] = uu;
        } else {
            // bond at row r-1: (u_{r-1}, m_r); c[0] = u_{r-1} before the
            // layer, c[1] = m_{r-1} after it
            T2 uu = c[0], mm = m;
            bond_rot2<PO, G>(uu, mm, k, a_moved);
            qu = uu;
            qm = c[1];
            c[0] = u;
            c[1] = mm;
        }
    }

    template <int PH>
    __device__ __forceinline__ void iter(int J, int st_lo, unsigned st_n, uint32_t lo_ok,
                                         uint32_t hi_ok, float *out_lo, float *out_hi) {
        constexpr int S0 = PH, S1 = (PH + 3) & 3, S2 = (PH + 2) & 3, S3 = (PH + 1) & 3;
        // every lane is done with the slot of row J - 1 before it is refilled
        __syncwarp();
        stage<(PH + 3) & (NSLOT - 1)>();
        cp_async_wait<NSLOT - 2>();
        // row J + 1, copied by all lanes, is complete and visible
        __syncwarp();
        const Slot &sl = ring[PH];
        float l2 = sl.q[0][lane], h2 = sl.q[0][lane + 32];
        float l3 = sl.q[1][lane], h3 = sl.q[1][lane + 32];
        float l4 = sl.q[2][lane], h4 = sl.q[2][lane + 32];
        if constexpr (VIN && !UNI) {
            if (vlive_lo) potential(l2, l3, l4, vlo);
            if (vlive_hi) potential(h2, h3, h4, vhi);
        }
        T2 q2 = PO::make(l2, h2), q3 = PO::make(l3, h3), q4 = PO::make(l4, h4);

        const K2<PO> &k0 = ring_coef<S0>();
        ux_layer<0>(q2, q4, k0);
        ux_layer<1>(q2, q4, k0);
        ux_layer<2>(q2, q4, k0);
        ux_layer<3>(q2, q4, k0);
        ux_layer<4>(q2, q4, k0);
        ux_layer<5>(q2, q4, k0);
        ux_layer<6>(q2, q4, k0);
        ux_layer<7>(q2, q4, k0);

        // q4 (untouched by U_y) is final for row J
        if (unsigned(J - st_lo) < st_n) {
            if (lo_ok) out_lo[2 * plane + o_now] = PO::lo(q4);
            if (hi_ok) out_hi[2 * plane + o_now] = PO::hi(q4);
        }
        o_now = next_row(o_now);

        uy_local<0>(q2, q3, ring_coef<S0>());                  // L1, row J
        uy_neighbour<1>(q2, q3, carry[0], ring_coef<S0>());    // L2 -> row J-1
        uy_local<2>(q2, q3, ring_coef<S1>());                  // L3, row J-1
        uy_neighbour<3>(q2, q3, carry[1], ring_coef<S2>());    // L4 -> row J-2
        uy_local<4>(q2, q3, ring_coef<S2>());                  // L5, row J-2
        uy_neighbour<5>(q2, q3, carry[2], ring_coef<S3>());    // L6 -> row J-3
        uy_local<6>(q2, q3, ring_coef<S3>());                  // L7, row J-3
        uy_neighbour<7>(q2, q3, carry[3], ring_coef<S3>());    // L8 -> row J-4
        // row J - 3's coefficients are dead: row J + 1's go into that slot
        if constexpr (!UNI) lookup_next<(PH + 1) & (NSLOT - 1), S3>();

        // q2, q3 of row J - 4 are final
        if (unsigned(J - LAG - st_lo) < st_n) {
            if (lo_ok) {
                out_lo[o_out] = PO::lo(q2);
                out_lo[plane + o_out] = PO::lo(q3);
            }
            if (hi_ok) {
                out_hi[o_out] = PO::hi(q2);
                out_hi[plane + o_out] = PO::hi(q3);
            }
        }
        o_out = next_row(o_out);
    }

    // The row in staging slot S, with the pending V applied (VIN).
    // The reads are volatile: a value read here may only be used in the next
    // iteration (q3 waits there for U_y), and the read must not sink past the
    // next iteration's copy into this slot.
    template <int S>
    __device__ __forceinline__ void load_row(T2 &q2, T2 &q3, T2 &q4) {
        const volatile float(*sq)[W] = ring[S].q;
        float l2 = sq[0][lane], h2 = sq[0][lane + 32];
        float l3 = sq[1][lane], h3 = sq[1][lane + 32];
        float l4 = sq[2][lane], h4 = sq[2][lane + 32];
        if constexpr (VIN) {
            if (vlive_lo) potential(l2, l3, l4, vlo);
            if (vlive_hi) potential(h2, h3, h4, vhi);
        }
        q2 = PO::make(l2, h2);
        q3 = PO::make(l3, h3);
        q4 = PO::make(l4, h4);
    }

    __device__ __forceinline__ void store_q4(bool row_in, uint32_t lo_ok, uint32_t hi_ok,
                                             float *out_lo, float *out_hi, T2 q4) {
        if (row_in) {
            if (lo_ok) out_lo[2 * plane + o_now] = PO::lo(q4);
            if (hi_ok) out_hi[2 * plane + o_now] = PO::hi(q4);
        }
        o_now = next_row(o_now);
    }

    // Interleaved march, iteration J (PH = (J - J0) mod 4): U_x of row J + 1
    // and U_y of row J are independent, and their layers alternate in the
    // instruction stream, so each warp has two dependent chains to issue
    // from (a bond layer's shuffles no longer stall the warp).  Rows are
    // staged four ahead; on entry knext holds row J + 1's coefficients and
    // (p2, p3) row J after U_x.
    template <int PH>
    __device__ __forceinline__ void iter_ilv(int J, int st_lo, unsigned st_n, uint32_t lo_ok,
                                             uint32_t hi_ok, float *out_lo, float *out_hi) {
        constexpr int S0 = PH, S1 = (PH + 3) & 3, S2 = (PH + 2) & 3, S3 = (PH + 1) & 3;
        // row J's slot was last read in the previous iteration: stage row
        // J + 4 into it
        __syncwarp();
        stage<PH>();
        cp_async_wait<NSLOT - 2>();
        // rows J + 1 and J + 2, copied by all lanes, are complete and visible
        __syncwarp();
        T2 n2, n3, n4;
        load_row<(PH + 1) & 3>(n2, n3, n4);

        ux_layer<0>(n2, n4, knext);
        uy_local<0>(p2, p3, kring[S0]);                  // L1, row J
        ux_layer<1>(n2, n4, knext);
        uy_neighbour<1>(p2, p3, carry[0], kring[S0]);    // L2 -> row J-1
        ux_layer<2>(n2, n4, knext);
        uy_local<2>(p2, p3, kring[S1]);                  // L3, row J-1
        ux_layer<3>(n2, n4, knext);
        uy_neighbour<3>(p2, p3, carry[1], kring[S2]);    // L4 -> row J-2
        ux_layer<4>(n2, n4, knext);
        uy_local<4>(p2, p3, kring[S2]);                  // L5, row J-2
        ux_layer<5>(n2, n4, knext);
        uy_neighbour<5>(p2, p3, carry[2], kring[S3]);    // L6 -> row J-3
        ux_layer<6>(n2, n4, knext);
        uy_local<6>(p2, p3, kring[S3]);                  // L7, row J-3
        ux_layer<7>(n2, n4, knext);
        uy_neighbour<7>(p2, p3, carry[3], kring[S3]);    // L8 -> row J-4

        // q4 of row J + 1 is final after U_x; q2, q3 of row J - 4 after U_y
        store_q4(unsigned(J + 1 - st_lo) < st_n, lo_ok, hi_ok, out_lo, out_hi, n4);
        if (unsigned(J - LAG - st_lo) < st_n) {
            if (lo_ok) {
                out_lo[o_out] = PO::lo(p2);
                out_lo[plane + o_out] = PO::lo(p3);
            }
            if (hi_ok) {
                out_hi[o_out] = PO::hi(p2);
                out_hi[plane + o_out] = PO::hi(p3);
            }
        }
        o_out = next_row(o_out);
        // row J - 3's slot is free: row J + 1's coefficients move in (they
        // are the next iteration's S0); row J + 2's are looked up
        kring[S3].copy_from(knext);
        lookup_into<(PH + 2) & 3>(knext);
        p2 = n2;
        p3 = n3;
    }

    // Work item `item`: window item % n_wx, row segment item / n_wx.
    // Needs nx a multiple of 4 (16-byte chunks stay inside a row) and >= 64.
    __device__ __forceinline__ void run_item(int nx, int ny, int seg_h, int n_wx, int item,
                                             Slot *warp_ring) {
        lane = threadIdx.x & 31;
        prev = (lane + 31) & 31;
        next = (lane + 1) & 31;
        first = lane == 0 ? 0xffffffffu : 0u;
        last = lane == 31 ? 0xffffffffu : 0u;
        ring = warp_ring;
        const int wx = item % n_wx, wy = item / n_wx;
        const int x0 = wx * WOUT - 4;   // window columns [x0, x0 + 64), periodic
        // staging: chunk h = lane & 15 (window columns 4h .. 4h + 3) of the
        // arrays lane / 16 (q2 or q3) and 2 + lane / 16 (q4 or the indices)
        const int h = lane & 15, a0 = lane >> 4, a1 = 2 + a0;
        const int gc = wrap(x0 + 4 * h, nx);
        src0 = reinterpret_cast<const char *>(in + size_t(a0) * plane + gc);
        src1 = a1 == 3 ? reinterpret_cast<const char *>(midx + gc)
                       : reinterpret_cast<const char *>(in + size_t(a1) * plane + gc);
        dst0 = uint32_t(a0 * W * 4 + 16 * h);
        dst1 = uint32_t(a1 * W * 4 + 16 * h);
        idx_lane = a1 == 3;
        // output columns: window columns [4, 60) inside the lattice
        const int xlo = x0 + lane, xhi = x0 + 32 + lane;
        const uint32_t lo_ok = lane >= 4 && xlo < nx ? 1u : 0u;
        const uint32_t hi_ok = lane < 28 && xhi < nx ? 1u : 0u;
        float *out_lo = out + wrap(xlo, nx);
        float *out_hi = out + wrap(xhi, nx);
        const int y_lo = wy * seg_h;
        const int y_hi = min(ny, y_lo + seg_h);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            carry[a][0] = PO::make(0.0f, 0.0f);
            carry[a][1] = PO::make(0.0f, 0.0f);
        }
        // the ring slots of the rows before J0 are read by the first
        // iterations (their results only reach halo rows, never stored
        // ones); they must hold defined values all the same, or the
        // compiler may substitute any register for them
#pragma unroll
        for (int a = 0; a < LAG; ++a) {
            kring[a].ch = kring[a].sh = kring[a].cl = kring[a].sl = PO::make(0.0f, 0.0f);
        }
        if constexpr (VIN) {
            vlive_lo = vlive_hi = 0u;
        }
        const int J0 = y_lo - LAG;
        const int J1 = y_hi + LAG;  // exclusive
        const unsigned st_n = unsigned(y_hi - y_lo);
        o_in = uint32_t(wrap(J0, ny)) * uint32_t(pitch);
        o_now = o_in;
        o_out = uint32_t(wrap(J0 - LAG, ny)) * uint32_t(pitch);
        if constexpr (ILV) {
            // rows J0 .. J0 + 3 in flight; U_x of row J0 before the loop
            stage<0>();
            stage<1>();
            stage<2>();
            stage<3>();
            cp_async_wait<2>();
            __syncwarp();
            lookup_into<0>(knext);
            T2 n4;
            load_row<0>(p2, p3, n4);
            ux_layer<0>(p2, n4, knext);
            ux_layer<1>(p2, n4, knext);
            ux_layer<2>(p2, n4, knext);
            ux_layer<3>(p2, n4, knext);
            ux_layer<4>(p2, n4, knext);
            ux_layer<5>(p2, n4, knext);
            ux_layer<6>(p2, n4, knext);
            ux_layer<7>(p2, n4, knext);
            store_q4(unsigned(J0 - y_lo) < st_n, lo_ok, hi_ok, out_lo, out_hi, n4);
            kring[0].copy_from(knext);
            lookup_into<1>(knext);
            for (int J = J0; J < J1; J += 4) {
                iter_ilv<0>(J + 0, y_lo, st_n, lo_ok, hi_ok, out_lo, out_hi);
                iter_ilv<1>(J + 1, y_lo, st_n, lo_ok, hi_ok, out_lo, out_hi);
                iter_ilv<2>(J + 2, y_lo, st_n, lo_ok, hi_ok, out_lo, out_hi);
                iter_ilv<3>(J + 3, y_lo, st_n, lo_ok, hi_ok, out_lo, out_hi);
            }
        } else {
            stage<0>();
            stage<1>();
            stage<2>();
            cp_async_wait<2>();
            __syncwarp();
            if constexpr (!UNI) lookup_next<0, 0>();
            for (int J = J0; J < J1; J += 4) {
                iter<0>(J + 0, y_lo, st_n, lo_ok, hi_ok, out_lo, out_hi);
                iter<1>(J + 1, y_lo, st_n, lo_ok, hi_ok, out_lo, out_hi);
                iter<2>(J + 2, y_lo, st_n, lo_ok, hi_ok, out_lo, out_hi);
                iter<3>(J + 3, y_lo, st_n, lo_ok, hi_ok, out_lo, out_hi);
            }
        }
        cp_async_wait<0>();
        __syncwarp();
    }
};

}  // namespace march
}  // namespace qla
