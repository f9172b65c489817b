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

// Pair arithmetic.  Three forms of the same operations (one rounding per
// fma.rn / mul.rn on each half, so the results are bitwise equal):
//   PairF2: float2 values and the packed intrinsics (negation of an operand
//           is folded into the instruction);
//   PairB64: 64-bit registers and inline fma.rn.f32x2 / mul.rn.f32x2 (a pair
//           stays in one aligned register pair for its whole life); PTX has
//           no packed negation, so the sine pairs are kept in both signs;
//   PairMix: 64-bit storage, intrinsic arithmetic on float2 views.
struct PairF2 {
    using T = float2;
    static constexpr bool NEG_RING = false;
    __device__ static __forceinline__ T make(float lo, float hi) { return make_float2(lo, hi); }
    __device__ static __forceinline__ float lo(T v) { return v.x; }
    __device__ static __forceinline__ float hi(T v) { return v.y; }
    __device__ static __forceinline__ T fma(T a, T b, T c) { return __ffma2_rn(a, b, c); }
    __device__ static __forceinline__ T mul(T a, T b) { return __fmul2_rn(a, b); }
    __device__ static __forceinline__ T neg(T a) { return make_float2(-a.x, -a.y); }
};

struct PairB64 {
    using T = unsigned long long;
    static constexpr bool NEG_RING = true;
    __device__ static __forceinline__ T make(float lo, float hi) {
        T r;
        asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
        return r;
    }
    __device__ static __forceinline__ float lo(T v) {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
        return a;
    }
    __device__ static __forceinline__ float hi(T v) {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
        return b;
    }
    __device__ static __forceinline__ T fma(T a, T b, T c) {
        T d;
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
        return d;
    }
    __device__ static __forceinline__ T mul(T a, T b) {
        T d;
        asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
        return d;
    }
    __device__ static __forceinline__ T neg(T a) { return a ^ 0x8000000080000000ull; }
};

struct PairMix {
    using T = unsigned long long;
    static constexpr bool NEG_RING = false;
    __device__ static __forceinline__ float2 f2(T v) {
        float2 r;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
        return r;
    }
    __device__ static __forceinline__ T u(float2 v) {
        T r;
        asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
        return r;
    }
    __device__ static __forceinline__ T make(float lo, float hi) { return u(make_float2(lo, hi)); }
    __device__ static __forceinline__ float lo(T v) { return f2(v).x; }
    __device__ static __forceinline__ float hi(T v) { return f2(v).y; }
    __device__ static __forceinline__ T fma(T a, T b, T c) {
        return u(__ffma2_rn(f2(a), f2(b), f2(c)));
    }
    __device__ static __forceinline__ T mul(T a, T b) { return u(__fmul2_rn(f2(a), f2(b))); }
    __device__ static __forceinline__ T neg(T a) {
        const float2 v = f2(a);
        return u(make_float2(-v.x, -v.y));
    }
};

// Two-word collision coefficients of two columns: (c_hi, s_hi, c_lo, s_lo)
// of Coef<float>, one column per half; with NEG_RING also -s_hi, -s_lo.
template <typename PO> struct K2 {
    typename PO::T ch, sh, cl, sl;
    typename PO::T nsh, nsl;   // used with NEG_RING only
};

// (a, b) <- [[c, -G s], [G s, c]] (a, b) on both halves: per element the
// operations of rotate(float &, float &, float4, float) in the same order.
template <typename PO, int G>
__device__ __forceinline__ void rotate2(typename PO::T &a, typename PO::T &b, const K2<PO> &k) {
    using T = typename PO::T;
    T shp, slp, shn, sln;   // G s and -G s, high and low words
    if constexpr (PO::NEG_RING) {
        shp = G > 0 ? k.sh : k.nsh;
        slp = G > 0 ? k.sl : k.nsl;
        shn = G > 0 ? k.nsh : k.sh;
        sln = G > 0 ? k.nsl : k.sl;
    } else {
        shp = G > 0 ? k.sh : PO::neg(k.sh);
        slp = G > 0 ? k.sl : PO::neg(k.sl);
        shn = PO::neg(shp);
        sln = PO::neg(slp);
    }
    const T na = PO::fma(k.ch, a, PO::fma(shn, b, PO::fma(k.cl, a, PO::mul(sln, b))));
    const T nb = PO::fma(k.ch, b, PO::fma(shp, a, PO::fma(k.cl, b, PO::mul(slp, a))));
    a = na;
    b = nb;
}

template <typename PO, int G>
__device__ __forceinline__ void bond_rot2(typename PO::T &u, typename PO::T &m, const K2<PO> &k,
                                          bool a_moved) {
    if (a_moved) rotate2<PO, G>(m, u, k);
    else rotate2<PO, G>(u, m, k);
}

template <int VM, bool VIN, typename PO = PairF2>
struct March2 {
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
    bool first, last;        // lane 0, lane 31
    // the lane's two staging copies: global sources at row 0, shared
    // destinations as byte offsets inside a slot
    const char *src0, *src1;
    uint32_t dst0, dst1;

    T2 carry[4][2];          // U_y neighbour layers: [layer][value]
    K2<PO> kring[LAG];       // collision coefficients of the rows in flight
    float4 vlo, vhi;         // row J+1's potential coefficients (low, high column)
    bool vlive_lo, vlive_hi; // row J+1's sites have their own records
    uint32_t o_in, o_now, o_out;

    __device__ __forceinline__ uint32_t next_row(uint32_t o) const {
        o += uint32_t(pitch);
        return o == total ? 0u : o;
    }

    template <int S>
    __device__ __forceinline__ void stage() {
        unsigned char *base = reinterpret_cast<unsigned char *>(ring + S);
        cp_async<16>(base + dst0, src0 + 4ull * o_in);
        cp_async<16>(base + dst1, src1 + 4ull * o_in);
        cp_async_commit();
        o_in = next_row(o_in);
    }

    // Row J + 1's records (staging slot S) into coefficient ring slot K and
    // the potential coefficients.
    template <int S, int K>
    __device__ __forceinline__ void lookup_next() {
        const uint32_t il = ring[S].idx[lane], ih = ring[S].idx[lane + 32];
        const MedRec<float> *rl = table + il, *rh = table + ih;
        const float4 cl = rl->c, chh = rh->c;
        kring[K].ch = PO::make(cl.x, chh.x);
        kring[K].sh = PO::make(cl.y, chh.y);
        kring[K].cl = PO::make(cl.z, chh.z);
        kring[K].sl = PO::make(cl.w, chh.w);
        if constexpr (PO::NEG_RING) {
            kring[K].nsh = PO::make(-cl.y, -chh.y);
            kring[K].nsl = PO::make(-cl.w, -chh.w);
        }
        if constexpr (VIN) {
            vlive_lo = il >= uint32_t(UNIFORM_SLOTS);
            vlive_hi = ih >= uint32_t(UNIFORM_SLOTS);
            if (vlive_lo) vlo = rl->v;
            if (vlive_hi) vhi = rh->v;
        }
    }

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
                        __shfl_sync(0xffffffffu, last ? ml : mh, prev));
    }
    __device__ __forceinline__ T2 give_right(T2 mm) const {
        const float ml = PO::lo(mm), mh = PO::hi(mm);
        return PO::make(__shfl_sync(0xffffffffu, first ? mh : ml, next),
                        __shfl_sync(0xffffffffu, mh, next));
    }
    __device__ __forceinline__ T2 take_right(T2 m) const {
        const float ml = PO::lo(m), mh = PO::hi(m);
        return PO::make(__shfl_sync(0xffffffffu, first ? mh : ml, next),
                        __shfl_sync(0xffffffffu, mh, next));
    }
    __device__ __forceinline__ T2 give_left(T2 mm) const {
        const float ml = PO::lo(mm), mh = PO::hi(mm);
        return PO::make(__shfl_sync(0xffffffffu, ml, prev),
                        __shfl_sync(0xffffffffu, last ? ml : mh, prev));
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
    __device__ __forceinline__ void iter(int J, int st_lo, unsigned st_n, bool lo_ok,
                                         bool hi_ok, float *out_lo, float *out_hi) {
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
        if constexpr (VIN) {
            if (vlive_lo) potential(l2, l3, l4, vlo);
            if (vlive_hi) potential(h2, h3, h4, vhi);
        }
        T2 q2 = PO::make(l2, h2), q3 = PO::make(l3, h3), q4 = PO::make(l4, h4);

        const K2<PO> &k0 = kring[S0];
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

        uy_local<0>(q2, q3, kring[S0]);                  // L1, row J
        uy_neighbour<1>(q2, q3, carry[0], kring[S0]);    // L2 -> row J-1
        uy_local<2>(q2, q3, kring[S1]);                  // L3, row J-1
        uy_neighbour<3>(q2, q3, carry[1], kring[S2]);    // L4 -> row J-2
        uy_local<4>(q2, q3, kring[S2]);                  // L5, row J-2
        uy_neighbour<5>(q2, q3, carry[2], kring[S3]);    // L6 -> row J-3
        uy_local<6>(q2, q3, kring[S3]);                  // L7, row J-3
        uy_neighbour<7>(q2, q3, carry[3], kring[S3]);    // L8 -> row J-4
        // row J - 3's coefficients are dead: row J + 1's go into that slot
        lookup_next<(PH + 1) & (NSLOT - 1), S3>();

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

    // Work item `item`: window item % n_wx, row segment item / n_wx.
    // Needs nx a multiple of 4 (16-byte chunks stay inside a row) and >= 64.
    __device__ __forceinline__ void run_item(int nx, int ny, int seg_h, int n_wx, int item,
                                             Slot *warp_ring) {
        lane = threadIdx.x & 31;
        prev = (lane + 31) & 31;
        next = (lane + 1) & 31;
        first = lane == 0;
        last = lane == 31;
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
        // output columns: window columns [4, 60) inside the lattice
        const int xlo = x0 + lane, xhi = x0 + 32 + lane;
        const bool lo_ok = lane >= 4 && xlo < nx;
        const bool hi_ok = lane < 28 && xhi < nx;
        float *out_lo = out + wrap(xlo, nx);
        float *out_hi = out + wrap(xhi, nx);
        const int y_lo = wy * seg_h;
        const int y_hi = min(ny, y_lo + seg_h);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            carry[a][0] = PO::make(0.0f, 0.0f);
            carry[a][1] = PO::make(0.0f, 0.0f);
        }
        if constexpr (VIN) {
            vlive_lo = vlive_hi = false;
        }
        const int J0 = y_lo - LAG;
        const int J1 = y_hi + LAG;  // exclusive
        const unsigned st_n = unsigned(y_hi - y_lo);
        o_in = uint32_t(wrap(J0, ny)) * uint32_t(pitch);
        o_now = o_in;
        o_out = uint32_t(wrap(J0 - LAG, ny)) * uint32_t(pitch);
        stage<0>();
        stage<1>();
        stage<2>();
        cp_async_wait<2>();
        __syncwarp();
        lookup_next<0, 0>();
        for (int J = J0; J < J1; J += 4) {
            iter<0>(J + 0, y_lo, st_n, lo_ok, hi_ok, out_lo, out_hi);
            iter<1>(J + 1, y_lo, st_n, lo_ok, hi_ok, out_lo, out_hi);
            iter<2>(J + 2, y_lo, st_n, lo_ok, hi_ok, out_lo, out_hi);
            iter<3>(J + 3, y_lo, st_n, lo_ok, hi_ok, out_lo, out_hi);
        }
        cp_async_wait<0>();
        __syncwarp();
    }
};

}  // namespace march
}  // namespace qla
