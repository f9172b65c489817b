// Internal declarations of libqla: the context, the coefficient records and
// the device-side rotation helpers shared by the kernels.  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <type_traits>

#include "../../include/qla.h"

namespace qla {

// ----------------------------------------------------------------------------
// Amplitude numbering (Eq. 3b3) and plane mapping.  A context stores P live
// planes: P = 6 holds q0..q5 in order; P = 3 (E_z polarisation) holds
// q2, q3, q4 as planes 0, 1, 2.  Collisions and potential steps never couple
// the triple (q2, q3, q4) with (q0, q1, q5) (Eqs. 2e3, 2e8, 2e11, 2e12), so a
// kernel may also step one triple of a six-plane state in place: the plane
// sets P_TE6 (q2, q3, q4) and P_TM6 (q0, q1, q5), with the six-plane storage.
// plane_of<P>(c) is q_c's plane in storage, -1 for an absent q_c;
// slot_of<P>(c) its index among the set's nplanes<P>() planes.
// ----------------------------------------------------------------------------
constexpr int P_TE6 = 7, P_TM6 = 8;
template <int P>
__host__ __device__ constexpr int plane_of(int c) {
    return P == 6       ? c
         : P == 3       ? (c >= 2 && c <= 4 ? c - 2 : -1)
         : P == P_TE6   ? (c >= 2 && c <= 4 ? c : -1)
                        : (c == 0 || c == 1 || c == 5 ? c : -1);
}
template <int P> __host__ __device__ constexpr int nplanes() { return P == 6 ? 6 : 3; }
template <int P>
__host__ __device__ constexpr int slot_of(int c) {
    return P == 6 ? c : P == P_TM6 ? (c == 5 ? 2 : c) : c - 2;
}
// whether the set holds the E_z triple, the (q0, q1, q5) triple
template <int P> __host__ __device__ constexpr bool has_te() { return P != P_TM6; }
template <int P> __host__ __device__ constexpr bool has_tm() { return P == 6 || P == P_TM6; }

// ----------------------------------------------------------------------------
// The eight collisions of one evolution operator U (Eqs. 2e6, 2e9).
//
// Written as acting on Q, U = C^ S1- C S1+ | C^ S2+ C S2- | C S1+ C^ S1- |
// C S2- C^ S2+ (each group read left to right = order of action; S1 is S14
// along x, S03 along y; S2 is S25).  Inside a group the shifted component
// returns to its place after the second collision, so each group is a
// site-local collision followed by a collision of "bonds" that pair the
// unshifted component at site i with the shifted one at site i + sigma,
// rotated with the angle of site i.  No data moves: U is eight layers of
// disjoint 2x2 rotations.  Per layer: adjoint flag, which component of each
// pair is the shifted one (0 none, 1 the S1 mover, 2 the S25 mover), sigma.
// ----------------------------------------------------------------------------
struct Layer { int dag, mover, shift; };
__host__ __device__ constexpr Layer layer_of(int l) {
    return l == 0 ? Layer{1, 0, 0} : l == 1 ? Layer{0, 1, -1}
         : l == 2 ? Layer{1, 0, 0} : l == 3 ? Layer{0, 2, +1}
         : l == 4 ? Layer{0, 0, 0} : l == 5 ? Layer{1, 1, +1}
         : l == 6 ? Layer{0, 0, 0} : Layer{1, 2, -1};
}

// Pairs rotated by a collision.  a is the first component of the pair in
// the printed matrix (its row holds cos, -g sin), b the second; m1 is the
// component moved by S14 (x) or S03 (y), the other is moved by S25.
//   x (Eq. 2e3):  (q1, q5) with q1 = S14 mover;  (q2, q4) with q4 = S14 mover
//   y (Eq. 2e8):  (q0, q5) with q0 = S03 mover;  (q2, q3) with q3 = S03 mover
// Sign g of the sine: C_x rotates by +theta, C_y by -theta; adjoints flip.
struct Pair { int a, b; bool a_is_m1; };
__host__ __device__ constexpr Pair pair_of(bool xdir, int k) {
    return xdir ? (k == 0 ? Pair{1, 5, true} : Pair{2, 4, false})
                : (k == 0 ? Pair{0, 5, true} : Pair{2, 3, false});
}

// ----------------------------------------------------------------------------
// Coefficient records, one per site.
//   FP64: CoefC = (tan(theta/2), sin theta), the three-shear form of the
//         rotation (rotate below); CoefV = (cos phi_x, sin phi_x,
//         cos phi_y, sin phi_y) with phi = beta/2 (rotation reading) or beta
//         (printed shear).
//   FP32: CoefC = (c_hi, s_hi, c_lo, s_lo): cos theta and sin theta each
//         split into an FP32 value and the FP32 rounding of the remainder,
//         so the collision angle and norm carry ~48 bits (single FP32 words
//         would shift the phase speed by ~1e-7 per step and drift the norm);
//         CoefV = (gamma_x, s_x, gamma_y, s_y), gamma = 1 - cos, single words.
// ----------------------------------------------------------------------------
template <typename T> struct Coef;
template <> struct Coef<double> { using C = double2; using V = double4_16a; };
template <> struct Coef<float>  { using C = float4;  using V = float4; };

// Double-single amplitude: the unevaluated sum hi + lo of two FP32 words,
// |lo| <= ulp(hi) / 2 (Dekker's representation).  Stored as a float2 in the
// 8 bytes an FP64 amplitude occupies.
struct dsf {
    float hi, lo;
    dsf() = default;
    __host__ __device__ constexpr dsf(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dsf(int v) : hi(float(v)), lo(0.0f) {}
};
// A cosine and a sine as three FP32 words each, whose sums are the FP64
// values exactly (24 + 24 + 24 bits cover the 53 of a double).
struct alignas(16) DSCoef {
    float c0, s0, c1, s1, c2, s2, pad0, pad1;
};
struct DSCoefV {
    DSCoef x, y;    // V_x and V_y: cos and sin of the potential angles
};
template <> struct Coef<dsf> { using C = DSCoef; using V = DSCoefV; };

// Per-site medium record: collision and potential coefficients together.
// Sites whose four neighbours have the same n as the site itself (the bulk
// of any piecewise-uniform medium) share one record per distinct n; every
// other site (the boundary layers) has its own.  A 32-bit index per site
// selects the record, so a step reads 4 bytes of medium per site instead of
// the 32 (FP32) or 48 (FP64) bytes of a full record.
template <typename T> struct MedRec {
    typename Coef<T>::C c;
    typename Coef<T>::V v;
};
constexpr int UNIFORM_SLOTS = 4096;  // open-addressing slots for shared records

// 64-bit finaliser that spreads a key's bits before it picks a slot of the
// shared-record table (the key is the bit pattern of a site's n).
__device__ __forceinline__ unsigned long long mix64(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// (a, b) <- [[c, -g s], [g s, c]] (a, b) with g = +-1, as three shears:
// a -= g t b, b += g s a, a -= g t b with k = (t, s) = (tan(theta/2),
// sin theta).  The product of the shears is the rotation because
// 1 - t s = cos theta and t (2 - t s) = sin theta; its determinant is 1 for
// any rounded t and s.  Three FMAs instead of two products and two FMAs: the
// FP64 step is bound by the FP64 pipe.  Explicit FMAs fix the rounding, so
// every kernel produces the same bits.
__device__ __forceinline__ void rotate(double &a, double &b, double2 k, double g) {
    const double t = g * k.x, s = g * k.y;
    a = fma(-t, b, a);
    b = fma(s, a, b);
    a = fma(-t, b, a);
}

// Same rotation with two-word c and s: the low-word terms are accumulated
// first, then the sine term, and the cosine term last, so each output is
// rounded once at its own magnitude (plus once at the sine term's).
__device__ __forceinline__ void rotate(float &a, float &b, float4 k, float g) {
    const float sh = g * k.y, sl = g * k.w;
    const float na = fmaf(k.x, a, fmaf(-sh, b, fmaf(k.z, a, -sl * b)));
    const float nb = fmaf(k.x, b, fmaf(sh, a, fmaf(k.z, b, sl * a)));
    a = na;
    b = nb;
}

// Double-single rotation row: c x + gs y with c, s in three words and
// gs = +-1 folded into the sine.  The two leading products are exact
// (p + pe = c0 x.hi and q + qe = s0 y.hi by FMA); their sum is split
// exactly (Knuth's two-sum); every smaller term is accumulated in FP32 at
// the low word's scale, and the result renormalised (fast two-sum).  Error
// ~2^-48 of the inputs' magnitude, unbiased.
__device__ __forceinline__ dsf ds_row(const DSCoef &k, dsf x, float gs, dsf y) {
    const float s0 = gs * k.s0, s1 = gs * k.s1, s2 = gs * k.s2;
    const float p = k.c0 * x.hi, pe = fmaf(k.c0, x.hi, -p);
    const float q = s0 * y.hi, qe = fmaf(s0, y.hi, -q);
    const float h = p + q, hb = h - p;
    const float e = (p - (h - hb)) + (q - hb);
    float t = e + (pe + qe);
    t = fmaf(k.c0, x.lo, t);
    t = fmaf(k.c1, x.hi, t);
    t = fmaf(k.c1, x.lo, t);
    t = fmaf(k.c2, x.hi, t);
    t = fmaf(s0, y.lo, t);
    t = fmaf(s1, y.hi, t);
    t = fmaf(s1, y.lo, t);
    t = fmaf(s2, y.hi, t);
    const float r = h + t;
    return dsf(r, t - (r - h));
}

// (a, b) <- [[c, -g s], [g s, c]] (a, b) in double-single arithmetic.
__device__ __forceinline__ void rotate(dsf &a, dsf &b, const DSCoef &k, dsf g) {
    const dsf na = ds_row(k, a, -g.hi, b);
    const dsf nb = ds_row(k, b, g.hi, a);
    a = na;
    b = nb;
}

// Single-word rotation used for V in FP32: (gamma, s) = (1 - cos, sin).
__device__ __forceinline__ void rotate1(float &a, float &b, float gam, float s, float g) {
    const float sg = g * s;
    const float ta = fmaf(gam, a, sg * b);
    const float tb = fmaf(gam, b, -sg * a);
    a -= ta;
    b -= tb;
}
__device__ __forceinline__ void rotate1(double &a, double &b, double c, double s, double g) {
    const double sg = g * s;
    const double na = fma(c, a, -(sg * b));
    const double nb = fma(c, b, sg * a);
    a = na;
    b = nb;
}

// Printed shear row: y <- c y + g s x (only y changes).
__device__ __forceinline__ void shear1(float x, float &y, float gam, float s, float g) {
    y -= fmaf(gam, y, -g * s * x);
}
__device__ __forceinline__ void shear1(double x, double &y, double c, double s, double g) {
    y = fma(c, y, g * s * x);
}

enum VMode { V_ROTATION = 0, V_LITERAL = 1, V_NONE = 2, V_LCU = 3 };

// Cosine and sine of a potential angle from a CoefV entry pair: FP64 stores
// (cos, sin), FP32 (gamma = 1 - cos, sin).
__device__ __forceinline__ void cos_sin(double a, double b, double &c, double &s) { c = a; s = b; }
__device__ __forceinline__ void cos_sin(float a, float b, float &c, float &s) { c = 1.0f - a; s = b; }

// Eqs. 2f1-2f7: V = (1/2)(L1 + L2 + L3 + L4), each printed L applied to the
// six amplitudes and the four results summed row by row, then halved.
// (c0, s0), (c2, s2): V_x angles beta_0 (q1, q5) and beta_2 (q2, q4);
// (c1, s1), (c3, s3): V_y angles beta_1 (q0, q5) and beta_3 (q2, q3).
template <typename T>
__device__ __forceinline__ void lcu_x(T (&v)[6], T c0, T s0, T c2, T s2) {
    T o[6];
    o[0] = v[0] - v[0] + v[0] + v[0];
    o[1] = v[1] + v[1] + (c0 * v[1] - s0 * v[5]) + (-c0 * v[1] + s0 * v[5]);
    o[2] = v[2] + v[2] + (c2 * v[2] + s2 * v[4]) + (-c2 * v[2] - s2 * v[4]);
    o[3] = v[3] - v[3] + v[3] + v[3];
    o[4] = v[4] - v[4] + (-s2 * v[2] + c2 * v[4]) + (-s2 * v[2] + c2 * v[4]);
    o[5] = v[5] - v[5] + (s0 * v[1] + c0 * v[5]) + (s0 * v[1] + c0 * v[5]);
#pragma unroll
    for (int r = 0; r < 6; ++r) v[r] = T(0.5) * o[r];
}
template <typename T>
__device__ __forceinline__ void lcu_y(T (&v)[6], T c1, T s1, T c3, T s3) {
    T o[6];
    o[0] = v[0] + v[0] + (c1 * v[0] + s1 * v[5]) + (-c1 * v[0] - s1 * v[5]);
    o[1] = v[1] - v[1] + v[1] + v[1];
    o[2] = v[2] + v[2] + (-s3 * v[2] + c3 * v[3]) + (s3 * v[2] - c3 * v[3]);
    o[3] = v[3] - v[3] + (c3 * v[2] + s3 * v[3]) + (c3 * v[2] + s3 * v[3]);
    o[4] = v[4] - v[4] + v[4] + v[4];
    o[5] = v[5] - v[5] + (-s1 * v[0] + c1 * v[5]) + (-s1 * v[0] + c1 * v[5]);
#pragma unroll
    for (int r = 0; r < 6; ++r) v[r] = T(0.5) * o[r];
}

// Potential operators at one site: V_x then V_y (Eq. 2e14).  q[] holds the
// six amplitudes (entries absent in E_z mode are ignored).  kv = CoefV.
template <typename T, int P, int VM, typename KV>
__device__ __forceinline__ void apply_potential(T (&q)[6], KV kv) {
    constexpr bool te = has_te<P>(), tm = has_tm<P>();
    if constexpr (VM == V_ROTATION && std::is_same<T, dsf>::value) {
        // double-single: the same rotations with three-word cos and sin
        if constexpr (te) rotate(q[2], q[4], kv.x, T(-1));
        if constexpr (tm) rotate(q[1], q[5], kv.x, T(1));
        if constexpr (te) rotate(q[2], q[3], kv.y, T(1));
        if constexpr (tm) rotate(q[0], q[5], kv.y, T(-1));
    } else if constexpr (VM == V_ROTATION) {
        // V_x: (q2,q4) by [[c, s], [-s, c]]; (q1,q5) by [[c, -s], [s, c]]
        if constexpr (te) rotate1(q[2], q[4], kv.x, kv.y, T(-1));
        if constexpr (tm) rotate1(q[1], q[5], kv.x, kv.y, T(1));
        // V_y: (q2,q3) by [[c, -s], [s, c]]; (q0,q5) by [[c, s], [-s, c]]
        if constexpr (te) rotate1(q[2], q[3], kv.z, kv.w, T(1));
        if constexpr (tm) rotate1(q[0], q[5], kv.z, kv.w, T(-1));
    } else if constexpr (VM == V_LITERAL) {
        // V_x: q4 <- -sin q2 + cos q4; q5 <- +sin q1 + cos q5
        if constexpr (te) shear1(q[2], q[4], kv.x, kv.y, T(-1));
        if constexpr (tm) shear1(q[1], q[5], kv.x, kv.y, T(1));
        // V_y: q3 <- sin q2 + cos q3; q5 <- -sin q0 + cos q5
        if constexpr (te) shear1(q[2], q[3], kv.z, kv.w, T(1));
        if constexpr (tm) shear1(q[0], q[5], kv.z, kv.w, T(-1));
    } else if constexpr (VM == V_LCU) {
        T cx, sx, cy, sy;
        cos_sin(kv.x, kv.y, cx, sx);
        cos_sin(kv.z, kv.w, cy, sy);
        lcu_x(q, cx, sx, cx, sx);
        lcu_y(q, cy, sy, cy, sy);
    }
}

// Per-site record of a diagonal index tensor (six-plane contexts made with
// QLA_ANISOTROPIC): a collision coefficient per pair class and the potential
// coefficients of the E_z triple (from n_z) and of the (q0, q1, q5) triple
// (V_x from n_y, V_y from n_x), in the layouts of Coef<T>.
template <typename T> struct MedRecT {
    typename Coef<T>::C c15;   // C_x (q1, q5): theta_1 = delta/(4 n_y)
    typename Coef<T>::C c2;    // C_x (q2, q4) and C_y (q2, q3): theta_2 = delta/(4 n_z)
    typename Coef<T>::C c05;   // C_y (q0, q5): theta_0 = delta/(4 n_x)
    typename Coef<T>::V vz;    // V_x (q2, q4) from beta_2, V_y (q2, q3) from beta_3
    typename Coef<T>::V vt;    // V_x (q1, q5) from beta_0, V_y (q0, q5) from beta_1
};

// apply_potential with each pair's own coefficients (same operations, same
// order): kz for the pairs with q2, kt for the pairs with q5.
template <typename T, int P, int VM, typename KV>
__device__ __forceinline__ void apply_potential_tensor(T (&q)[6], KV kz, KV kt) {
    if constexpr (VM == V_ROTATION) {
        rotate1(q[2], q[4], kz.x, kz.y, T(-1));
        if constexpr (P == 6) rotate1(q[1], q[5], kt.x, kt.y, T(1));
        rotate1(q[2], q[3], kz.z, kz.w, T(1));
        if constexpr (P == 6) rotate1(q[0], q[5], kt.z, kt.w, T(-1));
    } else if constexpr (VM == V_LITERAL) {
        shear1(q[2], q[4], kz.x, kz.y, T(-1));
        if constexpr (P == 6) shear1(q[1], q[5], kt.x, kt.y, T(1));
        shear1(q[2], q[3], kz.z, kz.w, T(1));
        if constexpr (P == 6) shear1(q[0], q[5], kt.z, kt.w, T(-1));
    } else if constexpr (VM == V_LCU) {
        T c0, s0, c1, s1, c2, s2, c3, s3;
        cos_sin(kt.x, kt.y, c0, s0);
        cos_sin(kz.x, kz.y, c2, s2);
        cos_sin(kt.z, kt.w, c1, s1);
        cos_sin(kz.z, kz.w, c3, s3);
        lcu_x(q, c0, s0, c2, s2);
        lcu_y(q, c1, s1, c3, s3);
    }
}

// The six amplitudes of the state at site g (storage offset), with the
// pending potential operator applied when vin (entries absent in E_z mode
// are zero).
template <typename T, int P, int VM>
__device__ __forceinline__ void load_site(const T *q, size_t plane, size_t g, bool vin,
                                          const uint32_t *midx, const MedRec<T> *table,
                                          T (&s)[6]) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const int p = plane_of<P>(c);
        s[c] = p >= 0 ? q[p * plane + g] : T(0);
    }
    if constexpr (VM != V_NONE)
        if (vin) apply_potential<T, P, VM>(s, table[midx[g]].v);
}

__host__ __device__ inline int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

}  // namespace qla

// ----------------------------------------------------------------------------
// Context.
// ----------------------------------------------------------------------------
struct qla_ctx {
    int nx = 0, ny = 0, pitch = 0;  // pitch: elements per stored row
    double delta = 1.0;
    int prec = 0;                   // qla_precision
    unsigned flags = 0;
    int P = 6;                      // live planes
    int vmode = 0;                  // qla::VMode
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    bool owns_ws = false;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    void *state[2] = {nullptr, nullptr};
    int cur = 0;
    size_t plane_elems = 0;         // ny * pitch
    uint32_t *midx = nullptr;       // record index per site (ny * pitch)
    void *table = nullptr;          // MedRec<T>[UNIFORM_SLOTS + nx*ny]
    unsigned long long *keys = nullptr;  // UNIFORM_SLOTS hash keys (n bits)
    unsigned *counter = nullptr;    // records handed to non-uniform sites
    int march_lx = 0, march_seg = 0;  // tuning (0 = automatic)
    double *n = nullptr;            // ny * pitch (n_z of a tensor medium)
    // QLA_ANISOTROPIC contexts: n_x, n_y planes (ny * pitch) and, with six
    // planes, one MedRecT<T> per stored site (indexed like the state)
    bool tensor = false;
    double *n_x = nullptr, *n_y = nullptr;
    void *ttable = nullptr;
    // QLA_DOUBLE_SINGLE contexts: MedRec<dsf> records, indexed like table
    void *dstable = nullptr;
    double *staging = nullptr;      // ny * nx
    double *partials = nullptr;     // energy partial sums
    double *result = nullptr;       // final energy (device)
    int energy_blocks = 0;
    bool has_medium = false, has_state = false;
    // True once a step has run since the state was last set: the buffer then
    // holds U_y U_x Q of the last step and the state Q itself is V applied to
    // it (the step kernels apply that V to their input; read-outs apply it
    // on the fly with the same device code).
    bool pending_v = false;
    int step_kernel = 0;            // qla_step_kernel
    long long launches = 0;
    // FP32 E_z contexts: the plateau-split step's unit list (workspace,
    // items_cap int4 entries) and the plan it holds, valid for the medium
    // of set_medium call number medium_gen and the given segment height
    long long medium_gen = 0;
    int *items = nullptr;
    size_t items_cap = 0;
    struct {
        long long gen = -1;
        int seg = 0, n_items = 0, n_list = 0, n_uniform = 0, n_sets = 0;
        // dataflow plan (units in item order; byte offsets into items of
        // the two dependency tables and of the counters: the hand-out
        // counter, then one per item from off_ctr + 16)
        bool flow = false, want_flow = false;
        int n_wx = 0, shift = 0;
        size_t off_xdep = 0, off_ydep = 0, off_ctr = 0;
    } uplan;
    // dataflow steps: a launch whose wait flag has not been read yet, each
    // wait's limit in SM cycles, and a test hook (the handed-out unit index
    // whose completion is withheld, -1 none)
    bool flow_unchecked = false;
    long long flow_budget = 1LL << 32;
    long long flow_withhold = -1;
    qla_status sticky = QLA_OK;
    std::string err;
};

namespace qla {
// Workspace layout: offsets of each region (bytes, 256-aligned).
struct Layout {
    size_t state[2], midx, table, keys, counter, n, staging, partials, result, total;
    size_t n_x, n_y, ttable;  // QLA_ANISOTROPIC only (else 0)
    size_t dstable;           // QLA_DOUBLE_SINGLE only (else 0)
    size_t items, items_cap;  // FP32 E_z only (else 0): marching work-item list
    size_t plane_elems;
    int pitch, energy_blocks;
};
Layout layout_for(int nx, int ny, int prec, unsigned flags);

// Launchers (host), each returns the cudaError_t of its launch.
cudaError_t launch_medium(qla_ctx *c);
// Tensor media: stage one host plane (already in c->staging) into dst;
// build the MedRecT table of a six-plane QLA_ANISOTROPIC context.
cudaError_t launch_pitch_copy(qla_ctx *c, double *dst);
// Raw forms for a six-plane state without a pending V (three dimensions:
// rows = ny * nz).  Each returns the cudaError_t of its launches.
cudaError_t raw_pitch_copy(const double *src, double *dst, int nx, int rows, int pitch,
                           cudaStream_t st);
cudaError_t raw_from_f64(int prec, const double *src, void *plane, int nx, int rows, int pitch,
                         cudaStream_t st);
cudaError_t raw_to_f64(int prec, const void *state, size_t plane_elems, int comp, double *dst,
                       int nx, int rows, int pitch, cudaStream_t st);
cudaError_t raw_energy(int prec, const void *state, size_t plane_elems, int nx, int rows,
                       int pitch, double *partials, int nblocks, double *result, cudaStream_t st);
cudaError_t launch_medium_tensor(qla_ctx *c);
cudaError_t launch_step_tensor(qla_ctx *c, const void *in, void *out);
// QLA_DOUBLE_SINGLE: the marching step on word-pair state with the
// double-single records, and the in-place conversions of the state buffer
// between FP64 and word pairs.
cudaError_t launch_step_march_ds(qla_ctx *c, const void *in, void *out, bool vin);
int step_march_ds_launches(const qla_ctx *c);   // kernels one such step launches
cudaError_t launch_state_to_ds(qla_ctx *c, void *state);
cudaError_t launch_state_from_ds(qla_ctx *c, void *state);
// Lattices the double-single step takes (those of the FP64 marching kernel).
bool ds_shape_ok(int nx, int ny);
// n FP64 values <-> n (hi, lo) FP32 word pairs, in place.
cudaError_t raw_to_ds(void *q, size_t n, cudaStream_t st);
cudaError_t raw_from_ds(void *q, size_t n, cudaStream_t st);
cudaError_t launch_packet(qla_ctx *c, const qla_packet &p);
cudaError_t launch_from_f64(qla_ctx *c, int plane, const double *src);
cudaError_t launch_to_f64(qla_ctx *c, int comp, double *dst);
cudaError_t launch_fields(qla_ctx *c, int comp, double *dst);
cudaError_t launch_energy(qla_ctx *c);
// Gauss-law monitors (Eqs. 3.1, 3.2): sums of (div B)^2, (d_x B_x)^2 +
// (d_y B_y)^2, (div D)^2, the D scale, then max |div B|, max |div D|.
constexpr int DIV_TERMS = 6;
cudaError_t launch_divergence(qla_ctx *c);
cudaError_t launch_probe(qla_ctx *c, int count, const int *ij_dev, double *out_dev);
cudaError_t launch_step_tile(qla_ctx *c, const void *in, void *out, bool vin);
// Domain decomposition: copy a rectangle of the stored state (every live
// plane) into a contiguous buffer (to_box) or back; the energy of a
// rectangle into c->result; a packet on a window of a larger lattice.
cudaError_t launch_box_copy(qla_ctx *c, int i0, int j0, int w, int h, void *box, bool to_box);
cudaError_t launch_energy_box(qla_ctx *c, int i0, int j0, int w, int h);
cudaError_t launch_packet_window(qla_ctx *c, const qla_packet &p, int i0, int j0, int gnx,
                                 int gny);
cudaError_t launch_step_march(qla_ctx *c, const void *in, void *out, bool vin);
// Dataflow steps (FP32 E_z plateau split): n_steps steps of c->state[c->cur]
// in one persistent launch, leaving the result in state[c->cur ^ (n_steps &
// 1)].  *done = false (nothing enqueued) where the context does not take
// them; needs a pending potential step if the context has a potential.
cudaError_t launch_step_flow(qla_ctx *c, long long n_steps, bool *done);
// Reads (and clears) the wait flag of the dataflow launches since the last
// read; the stream must be idle.  Returns true if a wait ran out.
cudaError_t flow_timed_out(qla_ctx *c, bool *timed_out);
bool march_supported(const qla_ctx *c);
int march_lane_cols(const qla_ctx *c);
}  // namespace qla
