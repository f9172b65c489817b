// Three-dimensional QLA step: Q <- V_z V_y V_x U_z U_y U_x Q, with U_z and
// V_z read off Eq. 3b4 (see include/qla.h).  Three step kernels: three
// launches, one per axis (the FP64 default); the fused march along z (one
// launch; measured slower on 256^3: its per-plane barriers dominate); and
// the 2D march on every slice plus a column pipeline along z (the FP32
// default), both further below.  The per-axis form: a CTA stages 32 lines x 40 cells along the active axis (32
// outputs and a 4-cell periodic halo on each side, the reach of U) of all
// six planes and of the collision coefficients in shared memory, applies
// the eight bond layers of that axis's U (the layer form of Eq. 2e6, see
// layer_of), and writes the 32 inner cells of each line; the z pass then
// applies V_x, V_y, V_z to its outputs.  Three passes read and write the
// state three times per step: the simple form of the 3D path.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <new>
#include <string>

#include "qla_internal.h"
#include "qla_march.cuh"

namespace qla {
namespace {

constexpr int SEG = 32, HALO3 = 4, AX = SEG + 2 * HALO3, TB = 32, THREADS3 = 256;

// Pairs rotated by the collision of each axis: (a, b, a is the first-type
// mover).  x: Eq. 2e3, y: Eq. 2e8, z: the reading of Eq. 3b4.
__host__ __device__ constexpr Pair pair3_of(int axis, int k) {
    return axis == 0 ? (k == 0 ? Pair{1, 5, true} : Pair{2, 4, false})
         : axis == 1 ? (k == 0 ? Pair{0, 5, true} : Pair{2, 3, false})
                     : (k == 0 ? Pair{0, 4, true} : Pair{1, 3, false});
}

// Collision sign of layer L of U_z: C_z rotates by +theta (the sign pattern
// of C_x); the adjoint flips it.
template <int L> __host__ __device__ constexpr int layer_sign_z() {
    return layer_of(L).dag ? -1 : 1;
}

// Potential coefficients of one site for x, y, z, in the CoefV convention
// (FP64 (cos, sin), FP32 (gamma = 1 - cos, sin)).
template <typename T> struct V3 { T gx, sx, gy, sy, gz, sz; };
// Double-single (QLA_DOUBLE_SINGLE): cos and sin of each axis's angle as
// three FP32 words (their sums are the FP64 values).
template <> struct V3<dsf> { DSCoef x, y, z; };

// FP64 collision coefficients: (tan(theta/2), sin theta), three shears.
__device__ __forceinline__ void coef_c(double th, double2 &k) {
    k = make_double2(tan(0.5 * th), sin(th));
}
__device__ __forceinline__ void split2(double v, float &hi, float &lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - double(hi));
}
__device__ __forceinline__ void coef_c(double th, float4 &k) {
    double s, c;
    sincos(th, &s, &c);
    split2(c, k.x, k.z);
    split2(s, k.y, k.w);
}
__device__ __forceinline__ void split3(double v, float &a, float &b, float &c) {
    a = __double2float_rn(v);
    const double r = v - double(a);
    b = __double2float_rn(r);
    c = __double2float_rn(r - double(b));
}
__device__ __forceinline__ void coef_ds(double ph, DSCoef &k) {
    double s, c;
    sincos(ph, &s, &c);
    split3(c, k.c0, k.c1, k.c2);
    split3(s, k.s0, k.s1, k.s2);
    k.pad0 = k.pad1 = 0.0f;
}
__device__ __forceinline__ void coef_v(double ph, double &g, double &s) {
    g = cos(ph);
    s = sin(ph);
}
__device__ __forceinline__ void coef_v(double ph, float &g, float &s) {
    const double h = sin(0.5 * ph);
    g = __double2float_rn(2.0 * h * h);
    s = __double2float_rn(sin(ph));
}

__host__ __device__ inline size_t at3(int x, int y, int z, int ny, int pitch) {
    return (size_t(z) * ny + y) * size_t(pitch) + x;
}

template <typename T>
__global__ void k3_medium(const double *__restrict__ n, int nx, int ny, int nz, int pitch,
                          double delta, double vscale, typename Coef<T>::C *__restrict__ kc,
                          V3<T> *__restrict__ kv) {
    const size_t N = size_t(nx) * ny * nz;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int x = int(t % nx), y = int((t / nx) % ny), z = int(t / (size_t(nx) * ny));
        const size_t g = at3(x, y, z, ny, pitch);
        const double nn = n[g];
        const double bx = (n[at3(wrap(x + 1, nx), y, z, ny, pitch)] -
                           n[at3(wrap(x - 1, nx), y, z, ny, pitch)]) /
                          (2.0 * delta) / (nn * nn) * delta * delta;
        const double by = (n[at3(x, wrap(y + 1, ny), z, ny, pitch)] -
                           n[at3(x, wrap(y - 1, ny), z, ny, pitch)]) /
                          (2.0 * delta) / (nn * nn) * delta * delta;
        const double bz = (n[at3(x, y, wrap(z + 1, nz), ny, pitch)] -
                           n[at3(x, y, wrap(z - 1, nz), ny, pitch)]) /
                          (2.0 * delta) / (nn * nn) * delta * delta;
        typename Coef<T>::C c;
        coef_c(delta / (4.0 * nn), c);
        kc[g] = c;
        V3<T> v;
        coef_v(vscale * bx, v.gx, v.sx);
        coef_v(vscale * by, v.gy, v.sy);
        coef_v(vscale * bz, v.gz, v.sz);
        kv[g] = v;
    }
}

// Global coordinates of staged cell (a along the axis, b across it) of the
// CTA's tile; false if the line lies outside the lattice.
template <int AXIS>
__device__ __forceinline__ bool cell(int a, int b, int nx, int ny, int nz, int &x, int &y,
                                     int &z) {
    if constexpr (AXIS == 0) {
        x = wrap(int(blockIdx.x) * SEG - HALO3 + a, nx);
        y = int(blockIdx.y) * TB + b;
        z = int(blockIdx.z);
        return y < ny;
    } else if constexpr (AXIS == 1) {
        x = int(blockIdx.x) * TB + b;
        y = wrap(int(blockIdx.y) * SEG - HALO3 + a, ny);
        z = int(blockIdx.z);
        return x < nx;
    } else {
        x = int(blockIdx.x) * TB + b;
        y = int(blockIdx.z);
        z = wrap(int(blockIdx.y) * SEG - HALO3 + a, nz);
        return x < nx;
    }
}

// Shared-memory row stride: the x pass stages lines along x, and one
// padding column keeps its column-wise accesses off a single bank.
template <int AXIS> constexpr int LD = AXIS == 0 ? TB + 1 : TB;

template <typename T, int AXIS, bool VEND, int VM>
__global__ void __launch_bounds__(THREADS3)
k3_pass(const T *__restrict__ in, T *__restrict__ out, const typename Coef<T>::C *__restrict__ kc,
        const V3<T> *__restrict__ kv, int nx, int ny, int nz, int pitch, size_t plane_elems) {
    using CC = typename Coef<T>::C;
    constexpr int ld = LD<AXIS>, cells = AX * ld;
    extern __shared__ __align__(16) unsigned char smem3[];
    CC *sc = reinterpret_cast<CC *>(smem3);
    T *s = reinterpret_cast<T *>(sc + cells);
    // stage: consecutive threads take consecutive x
    for (int t = threadIdx.x; t < AX * TB; t += THREADS3) {
        const int a = AXIS == 0 ? t % AX : t / TB, b = AXIS == 0 ? t / AX : t % TB;
        int x, y, z;
        if (!cell<AXIS>(a, b, nx, ny, nz, x, y, z)) continue;
        const size_t g = at3(x, y, z, ny, pitch);
        const int i = a * ld + b;
#pragma unroll
        for (int c = 0; c < 6; ++c) s[c * cells + i] = in[c * plane_elems + g];
        sc[i] = kc[g];
    }
    __syncthreads();
    // the eight bond layers of this axis (Eq. 2e6 / 2e9 / their z analogue)
#pragma unroll
    for (int L = 0; L < 8; ++L) {
        const Layer ly = layer_of(L);
        const T g0 = T(AXIS == 1 ? -1 : 1);
        const T g = ly.dag ? -g0 : g0;
        for (int t = threadIdx.x; t < AX * TB; t += THREADS3) {
            const int a = t / TB, b = t % TB;
            const int a2 = a + ly.shift;
            if (a2 < 0 || a2 >= AX) continue;
            const int i = a * ld + b, i2 = a2 * ld + b;
#pragma unroll
            for (int pk = 0; pk < 2; ++pk) {
                const Pair pr = pair3_of(AXIS, pk);
                int ia = i, ib = i;
                if (ly.mover == 1) {
                    if (pr.a_is_m1) ia = i2; else ib = i2;
                } else if (ly.mover == 2) {
                    if (pr.a_is_m1) ib = i2; else ia = i2;
                }
                T va = s[pr.a * cells + ia], vb = s[pr.b * cells + ib];
                rotate(va, vb, sc[i], g);
                s[pr.a * cells + ia] = va;
                s[pr.b * cells + ib] = vb;
            }
        }
        __syncthreads();
    }
    // write the 32 inner cells of each line
    const int seg0 = int(AXIS == 0 ? blockIdx.x : blockIdx.y) * SEG;
    const int n_along = AXIS == 0 ? nx : AXIS == 1 ? ny : nz;
    for (int t = threadIdx.x; t < SEG * TB; t += THREADS3) {
        const int a = HALO3 + (AXIS == 0 ? t % SEG : t / TB), b = AXIS == 0 ? t / SEG : t % TB;
        if (seg0 + a - HALO3 >= n_along) continue;
        int x, y, z;
        if (!cell<AXIS>(a, b, nx, ny, nz, x, y, z)) continue;
        const size_t g = at3(x, y, z, ny, pitch);
        const int i = a * ld + b;
        T q[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) q[c] = s[c * cells + i];
        if constexpr (VEND && VM == V_ROTATION) {
            // V_x (Eq. 2e11, rotation reading), V_y (Eq. 2e12), V_z (Eq. 3b4)
            const V3<T> v = kv[g];
            rotate1(q[2], q[4], v.gx, v.sx, T(-1));
            rotate1(q[1], q[5], v.gx, v.sx, T(1));
            rotate1(q[2], q[3], v.gy, v.sy, T(1));
            rotate1(q[0], q[5], v.gy, v.sy, T(-1));
            rotate1(q[1], q[3], v.gz, v.sz, T(-1));
            rotate1(q[0], q[4], v.gz, v.sz, T(1));
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) out[c * plane_elems + g] = q[c];
    }
}

template <typename T, int AXIS, bool VEND, int VM>
cudaError_t pass_t(const void *in, void *out, const void *kc, const void *kv, int nx, int ny,
                   int nz, int pitch, size_t plane_elems, cudaStream_t st) {
    constexpr int cells = AX * LD<AXIS>;
    const size_t smem = size_t(cells) * (sizeof(typename Coef<T>::C) + 6 * sizeof(T));
    auto kern = k3_pass<T, AXIS, VEND, VM>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [&] {
        attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    });
    if (attr != cudaSuccess) return attr;
    dim3 grid;
    if (AXIS == 0) grid = dim3((nx + SEG - 1) / SEG, (ny + TB - 1) / TB, nz);
    else if (AXIS == 1) grid = dim3((nx + TB - 1) / TB, (ny + SEG - 1) / SEG, nz);
    else grid = dim3((nx + TB - 1) / TB, (nz + SEG - 1) / SEG, ny);
    kern<<<grid, THREADS3, smem, st>>>(static_cast<const T *>(in), static_cast<T *>(out),
                                       static_cast<const typename Coef<T>::C *>(kc),
                                       static_cast<const V3<T> *>(kv), nx, ny, nz, pitch,
                                       plane_elems);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused step: a CTA owns a TX x TY tile of (x, y) sites and marches along z
// over a segment of planes.  Per input plane: stage the tile and a 4-cell
// halo in x and y (all six planes and the collision coefficients), apply
// U_x to every staged row and U_y to the tile's columns in shared memory;
// U_z then runs as a software pipeline along z in registers, per site (the
// pipeline of the 2D march kernel along y: each neighbour layer delays its
// output by one plane and carries two values per pair), so the output plane
// is four planes behind the input plane.  q2 and q5, which no z pair
// touches, wait in a four-plane register ring so that V_x V_y V_z see all
// six amplitudes of the output plane; then it is stored.  A segment reads
// four planes on each side that it does not store.
// ---------------------------------------------------------------------------
template <typename T> struct MTile;
template <> struct MTile<float>  { static constexpr int TX = 32, TY = 16; };
template <> struct MTile<double> { static constexpr int TX = 32, TY = 8; };

// One on-site U_z layer on a site's six amplitudes (pairs (q0, q4), (q1, q3)).
template <typename T, int L>
__device__ __forceinline__ void uz_local(T (&q)[6], typename Coef<T>::C k) {
    const T g = T(layer_sign_z<L>());
#pragma unroll
    for (int pk = 0; pk < 2; ++pk) {
        const Pair pr = pair3_of(2, pk);
        rotate(q[pr.a], q[pr.b], k, g);
    }
}

// One neighbour U_z layer: q holds the plane entering the stage and on
// return the plane leaving it (one plane earlier); c[pk][0..1] carry the
// values the layer keeps between planes (as uy_neighbour in the 2D march).
template <typename T, int L>
__device__ __forceinline__ void uz_neighbour(T (&q)[6], T (&c)[2][2], typename Coef<T>::C k) {
    constexpr Layer ly = layer_of(L);
    const T g = T(layer_sign_z<L>());
#pragma unroll
    for (int pk = 0; pk < 2; ++pk) {
        const Pair pr = pair3_of(2, pk);
        const bool a_moved = (ly.mover == 1) == pr.a_is_m1;
        const int cm = a_moved ? pr.a : pr.b, cu = a_moved ? pr.b : pr.a;
        const T u = q[cu], m = q[cm];
        if (ly.shift < 0) {
            // bond at this plane r: (u_r, m_{r-1}); c0 = m_{r-1} before the
            // layer, c1 = u_{r-1} after it
            T uu = u, mm = c[pk][0];
            if (a_moved) rotate(mm, uu, k, g); else rotate(uu, mm, k, g);
            q[cu] = c[pk][1];
            q[cm] = mm;
            c[pk][0] = m;
            c[pk][1] = uu;
        } else {
            // bond at plane r-1: (u_{r-1}, m_r); c0 = u_{r-1} before the
            // layer, c1 = m_{r-1} after it
            T uu = c[pk][0], mm = m;
            if (a_moved) rotate(mm, uu, k, g); else rotate(uu, mm, k, g);
            q[cu] = uu;
            q[cm] = c[pk][1];
            c[pk][0] = u;
            c[pk][1] = mm;
        }
    }
}

template <typename T, int VM>
struct March3 {
    using CC = typename Coef<T>::C;
    static constexpr int TX = MTile<T>::TX, TY = MTile<T>::TY;
    static constexpr int RX = TX + 2 * HALO3, RY = TY + 2 * HALO3, CELLS = RX * RY;
    static constexpr int SPT = TX * TY / THREADS3;   // inner sites per thread

    const T *in;
    T *out;
    const CC *kc;
    const V3<T> *kv;
    int nx, ny, nz, pitch;
    size_t plane_elems;
    int x0, y0, z_lo, z_hi;
    T *s;
    CC *sc;
    T carry[SPT][4][2][2];   // [site][neighbour layer][pair][value]
    CC kring[SPT][4];        // coefficients of the four planes in the U_z pipeline
    T dring[SPT][4][2];      // q2, q5 of the four planes in flight

    // One bond of layer L of axis AXIS between staged cells a (the bond
    // site) and b (its partner at a + shift), both pairs.
    template <int AXIS>
    __device__ __forceinline__ void bond3(int L, int a, int b, T g) {
        const Layer ly = layer_of(L);
#pragma unroll
        for (int pk = 0; pk < 2; ++pk) {
            const Pair pr = pair3_of(AXIS, pk);
            int ia = a, ib = a;
            if (ly.mover == 1) { if (pr.a_is_m1) ia = b; else ib = b; }
            else if (ly.mover == 2) { if (pr.a_is_m1) ib = b; else ia = b; }
            T va = s[pr.a * CELLS + ia], vb = s[pr.b * CELLS + ib];
            rotate(va, vb, sc[a], g);
            s[pr.a * CELLS + ia] = va;
            s[pr.b * CELLS + ib] = vb;
        }
    }

    // Input plane J; PH = (J - first plane) mod 4 selects the ring slots
    // (slot S0 holds plane J, and held plane J - 4 until this iteration).
    template <int PH>
    __device__ __forceinline__ void plane(int J) {
        constexpr int S0 = PH, S1 = (PH + 3) & 3, S2 = (PH + 2) & 3, S3 = (PH + 1) & 3;
        const int zJ = wrap(J, nz);
        __syncthreads();   // the previous plane's readers are done with s
        for (int t = threadIdx.x; t < CELLS; t += THREADS3) {
            const int r = t / RX, c = t - r * RX;
            const int gx = wrap(x0 - HALO3 + c, nx), gy = wrap(y0 - HALO3 + r, ny);
            const size_t g = at3(gx, gy, zJ, ny, pitch);
#pragma unroll
            for (int k = 0; k < 6; ++k) s[k * CELLS + t] = in[k * plane_elems + g];
            sc[t] = kc[g];
        }
        __syncthreads();
        // U_x on every staged row (Eq. 2e6)
#pragma unroll
        for (int L = 0; L < 8; ++L) {
            const Layer ly = layer_of(L);
            const T g = ly.dag ? T(-1) : T(1);
            for (int t = threadIdx.x; t < CELLS; t += THREADS3) {
                const int r = t / RX, i = t - r * RX, i2 = i + ly.shift;
                if (i2 < 0 || i2 >= RX) continue;
                bond3<0>(L, r * RX + i, r * RX + i2, g);
            }
            __syncthreads();
        }
        // U_y on the tile's columns (Eq. 2e9)
#pragma unroll
        for (int L = 0; L < 8; ++L) {
            const Layer ly = layer_of(L);
            const T g = ly.dag ? T(1) : T(-1);
            for (int t = threadIdx.x; t < TX * RY; t += THREADS3) {
                const int r = t / TX, i = HALO3 + (t - r * TX), r2 = r + ly.shift;
                if (r2 < 0 || r2 >= RY) continue;
                bond3<1>(L, r * RX + i, r2 * RX + i, g);
            }
            __syncthreads();
        }
        // U_z along the march, per inner site; the output is plane J - 4
        const bool store = J - HALO3 >= z_lo && J - HALO3 < z_hi;
        const int zo = wrap(J - HALO3, nz);
#pragma unroll
        for (int p = 0; p < SPT; ++p) {
            const int site = int(threadIdx.x) + p * THREADS3;
            const int ix = site % TX, iy = site / TX;
            const int sm = (iy + HALO3) * RX + ix + HALO3;
            T q[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) q[k] = s[k * CELLS + sm];
            kring[p][S0] = sc[sm];
            uz_local<T, 0>(q, kring[p][S0]);
            uz_neighbour<T, 1>(q, carry[p][0], kring[p][S0]);
            uz_local<T, 2>(q, kring[p][S1]);
            uz_neighbour<T, 3>(q, carry[p][1], kring[p][S2]);
            uz_local<T, 4>(q, kring[p][S2]);
            uz_neighbour<T, 5>(q, carry[p][2], kring[p][S3]);
            uz_local<T, 6>(q, kring[p][S3]);
            uz_neighbour<T, 7>(q, carry[p][3], kring[p][S3]);
            // q2, q5 of the output plane J - 4 come out of the ring; those of
            // plane J go in (the same slot)
            const T q2 = dring[p][S0][0], q5 = dring[p][S0][1];
            dring[p][S0][0] = q[2];
            dring[p][S0][1] = q[5];
            q[2] = q2;
            q[5] = q5;
            const int gx = x0 + ix, gy = y0 + iy;
            if (store && gx < nx && gy < ny) {
                const size_t g = at3(gx, gy, zo, ny, pitch);
                if constexpr (VM == V_ROTATION) {
                    // V_x (Eq. 2e11, rotation reading), V_y (Eq. 2e12), V_z (Eq. 3b4)
                    const V3<T> v = kv[g];
                    rotate1(q[2], q[4], v.gx, v.sx, T(-1));
                    rotate1(q[1], q[5], v.gx, v.sx, T(1));
                    rotate1(q[2], q[3], v.gy, v.sy, T(1));
                    rotate1(q[0], q[5], v.gy, v.sy, T(-1));
                    rotate1(q[1], q[3], v.gz, v.sz, T(-1));
                    rotate1(q[0], q[4], v.gz, v.sz, T(1));
                }
#pragma unroll
                for (int k = 0; k < 6; ++k) out[k * plane_elems + g] = q[k];
            }
        }
    }
};

template <typename T, int VM>
__global__ void __launch_bounds__(THREADS3)
k3_march(const T *__restrict__ in, T *__restrict__ out, const typename Coef<T>::C *__restrict__ kc,
         const V3<T> *__restrict__ kv, int nx, int ny, int nz, int pitch, size_t plane_elems,
         int seg) {
    using M = March3<T, VM>;
    extern __shared__ __align__(16) unsigned char smem3[];
    M m;
    m.in = in;
    m.out = out;
    m.kc = kc;
    m.kv = kv;
    m.nx = nx;
    m.ny = ny;
    m.nz = nz;
    m.pitch = pitch;
    m.plane_elems = plane_elems;
    m.x0 = int(blockIdx.x) * M::TX;
    m.y0 = int(blockIdx.y) * M::TY;
    m.z_lo = int(blockIdx.z) * seg;
    m.z_hi = min(nz, m.z_lo + seg);
    m.sc = reinterpret_cast<typename M::CC *>(smem3);
    m.s = reinterpret_cast<T *>(m.sc + M::CELLS);
#pragma unroll
    for (int p = 0; p < M::SPT; ++p)
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            m.dring[p][l][0] = m.dring[p][l][1] = T(0);
#pragma unroll
            for (int a = 0; a < 2; ++a) m.carry[p][l][a][0] = m.carry[p][l][a][1] = T(0);
        }
    // input planes z_lo - 4 .. z_hi + 3 (rounded up to a multiple of 4; the
    // extra planes are computed and not stored); output plane J - 4
    const int J0 = m.z_lo - HALO3, J1 = m.z_hi + HALO3;
    for (int J = J0; J < J1; J += 4) {
        m.template plane<0>(J);
        m.template plane<1>(J + 1);
        m.template plane<2>(J + 2);
        m.template plane<3>(J + 3);
    }
}

template <typename T, int VM>
cudaError_t march3_t(const void *in, void *out, const void *kc, const void *kv, int nx, int ny,
                     int nz, int pitch, size_t plane_elems, int num_sms, cudaStream_t st) {
    using M = March3<T, VM>;
    const size_t smem = size_t(M::CELLS) * (sizeof(typename Coef<T>::C) + 6 * sizeof(T));
    auto kern = k3_march<T, VM>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    static int per_sm = 1;
    std::call_once(once, [&] {
        attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (attr == cudaSuccess)
            attr = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS3, smem);
        if (per_sm < 1) per_sm = 1;
    });
    if (attr != cudaSuccess) return attr;
    const int tiles = ((nx + M::TX - 1) / M::TX) * ((ny + M::TY - 1) / M::TY);
    // about two waves of CTAs; at least 16 planes per segment so that the
    // 8 planes a segment reads but does not store stay a modest overhead
    const long long want = 2LL * per_sm * num_sms;
    int nseg = int((want + tiles - 1) / tiles);
    if (nseg < 1) nseg = 1;
    int seg = (nz + nseg - 1) / nseg;
    if (seg < 16) seg = 16;
    nseg = (nz + seg - 1) / seg;
    dim3 grid((nx + M::TX - 1) / M::TX, (ny + M::TY - 1) / M::TY, nseg);
    kern<<<grid, THREADS3, smem, st>>>(static_cast<const T *>(in), static_cast<T *>(out),
                                       static_cast<const typename Coef<T>::C *>(kc),
                                       static_cast<const V3<T> *>(kv), nx, ny, nz, pitch,
                                       plane_elems, seg);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Slices + column pipeline (kernel 2).  Launch 1 runs the 2D marching
// machinery of qla_march.cuh on every z slice at once (work item = slice,
// 64-column window, row segment): U_x in registers with warp shuffles, U_y
// as a register pipeline along y, no V.  It reads the records of k3_dedup
// through their per-site index.  Launch 2 gives each thread one (x, y) column
// and marches it along z: U_z as the same register pipeline (q2 and q5,
// which no z pair touches, wait four planes in a ring), then V_x V_y V_z,
// then the store.  Neither launch uses shared-memory layer passes or block
// barriers.
// ---------------------------------------------------------------------------
// PS: the planes stepped (6, or one triple of the six-plane storage: U_x and
// U_y never couple (q2, q3, q4) with (q0, q1, q5); U_z does, in launch 2).
template <typename T, int PS>
__global__ void __launch_bounds__(32 * march::WARPS)
k3_slices(const T *__restrict__ in, T *__restrict__ out, const uint32_t *__restrict__ midx,
          const MedRec<T> *__restrict__ table, int nx, int ny, int pitch, size_t plane_elems,
          int seg_h, int n_wx, int n_wy, long long n_items) {
    using M = march::March<T, PS, 2, V_NONE, false>;
    extern __shared__ __align__(16) unsigned char smem_s[];
    typename M::Slot *ring =
        reinterpret_cast<typename M::Slot *>(smem_s) + (threadIdx.x >> 5) * march::NSLOT;
    const long long item = (long long)blockIdx.x * march::WARPS + (threadIdx.x >> 5);
    if (item >= n_items) return;
    const long long per_slice = (long long)n_wx * n_wy;
    const int slice = int(item / per_slice), local = int(item - slice * per_slice);
    const size_t base = size_t(slice) * ny * size_t(pitch);
    M m;
    m.in = in + base;
    m.out = out + base;
    m.midx = midx + base;
    m.table = table;
    m.pitch = pitch;
    m.plane = uint32_t(plane_elems);
    m.total = uint32_t(ny) * uint32_t(pitch);
    m.run_item(nx, ny, seg_h, n_wx, local, ring);
}

template <typename T, int VM, int PD>
struct ZCol {
    static_assert(PD == 1 || PD == 2 || PD == 4, "the prefetch ring must divide the 4-plane unroll");
    using CC = typename Coef<T>::C;
    const T *in;
    T *out;
    const uint32_t *idx3;
    const MedRec<T> *rec;
    const V3<T> *rv;
    size_t col, zstride, plane_elems;
    int nz;
    T carry[4][2][2];
    CC kring[4];
    T dring[4][2];
    uint32_t iring[4];       // record index of the four planes in flight
    // the next PD input planes, loaded ahead in a ring (offset and z of the
    // next plane to load)
    T nq[PD][6];
    uint32_t nid[PD];
    size_t g_next;
    int z_next;
    // the output plane's offset and how many planes are still to be stored
    size_t g_out;
    int z_out, to_skip, to_store;

    __device__ __forceinline__ void fetch(int slot) {
#pragma unroll
        for (int k = 0; k < 6; ++k) nq[slot][k] = in[k * plane_elems + g_next];
        nid[slot] = idx3[g_next];
        g_next += zstride;
        if (++z_next == nz) {
            z_next = 0;
            g_next = col;
        }
    }

    template <int PH>
    __device__ __forceinline__ void plane() {
        constexpr int S0 = PH, S1 = (PH + 3) & 3, S2 = (PH + 2) & 3, S3 = (PH + 1) & 3;
        constexpr int F = PH % PD;
        T q[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) q[k] = nq[F][k];
        const uint32_t id = nid[F];
        kring[S0] = rec[id].c;
        fetch(F);
        uz_local<T, 0>(q, kring[S0]);
        uz_neighbour<T, 1>(q, carry[0], kring[S0]);
        uz_local<T, 2>(q, kring[S1]);
        uz_neighbour<T, 3>(q, carry[1], kring[S2]);
        uz_local<T, 4>(q, kring[S2]);
        uz_neighbour<T, 5>(q, carry[2], kring[S3]);
        uz_local<T, 6>(q, kring[S3]);
        uz_neighbour<T, 7>(q, carry[3], kring[S3]);
        const T q2 = dring[S0][0], q5 = dring[S0][1];
        const uint32_t io = iring[S0];
        dring[S0][0] = q[2];
        dring[S0][1] = q[5];
        iring[S0] = id;
        q[2] = q2;
        q[5] = q5;
        if (to_skip > 0) {
            --to_skip;
        } else if (to_store > 0) {
            --to_store;
            if constexpr (VM == V_ROTATION && std::is_same<T, dsf>::value) {
                // the same rotations in double-single arithmetic
                const V3<T> v = rv[io];
                rotate(q[2], q[4], v.x, T(-1));
                rotate(q[1], q[5], v.x, T(1));
                rotate(q[2], q[3], v.y, T(1));
                rotate(q[0], q[5], v.y, T(-1));
                rotate(q[1], q[3], v.z, T(-1));
                rotate(q[0], q[4], v.z, T(1));
            } else if constexpr (VM == V_ROTATION) {
                // V_x (Eq. 2e11, rotation reading), V_y (Eq. 2e12), V_z (Eq. 3b4)
                const V3<T> v = rv[io];
                rotate1(q[2], q[4], v.gx, v.sx, T(-1));
                rotate1(q[1], q[5], v.gx, v.sx, T(1));
                rotate1(q[2], q[3], v.gy, v.sy, T(1));
                rotate1(q[0], q[5], v.gy, v.sy, T(-1));
                rotate1(q[1], q[3], v.gz, v.sz, T(-1));
                rotate1(q[0], q[4], v.gz, v.sz, T(1));
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) out[k * plane_elems + g_out] = q[k];
            g_out += zstride;
            if (++z_out == nz) {
                z_out = 0;
                g_out = col;
            }
        }
    }
};

template <typename T, int VM, int PD>
__global__ void __launch_bounds__(128)
k3_zcol(const T *__restrict__ in, T *__restrict__ out, const uint32_t *__restrict__ idx3,
        const MedRec<T> *__restrict__ rec, const V3<T> *__restrict__ rv, int nx, int ny, int nz,
        int pitch, size_t plane_elems, int seg) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // threads past the last column have nothing to do (no barrier follows)
    if (t >= (long long)nx * ny) return;
    ZCol<T, VM, PD> m;
    const int x = int(t % nx), y = int(t / nx);
    m.in = in;
    m.out = out;
    m.idx3 = idx3;
    m.rec = rec;
    m.rv = rv;
    m.col = size_t(y) * pitch + x;
    m.zstride = size_t(ny) * pitch;
    m.plane_elems = plane_elems;
    m.nz = nz;
    const int z_lo = int(blockIdx.y) * seg, z_hi = min(nz, z_lo + seg);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        m.dring[l][0] = m.dring[l][1] = T(0);
        m.iring[l] = 0;
#pragma unroll
        for (int a = 0; a < 2; ++a) m.carry[l][a][0] = m.carry[l][a][1] = T(0);
    }
    // planes J0 .. J1-1 enter the pipeline; plane J leaves it at step J + HALO3,
    // so the first 2 HALO3 outputs are the halo and the next z_hi - z_lo stored
    const int J0 = z_lo - HALO3, J1 = z_hi + HALO3;
    m.z_next = wrap(J0, nz);
    m.g_next = m.col + size_t(m.z_next) * m.zstride;
    m.z_out = z_lo;
    m.g_out = m.col + size_t(z_lo) * m.zstride;
    m.to_skip = 2 * HALO3;
    m.to_store = z_hi - z_lo;
#pragma unroll
    for (int f = 0; f < PD; ++f) m.fetch(f);
    for (int J = J0; J < J1; J += 4) {
        m.template plane<0>();
        m.template plane<1>();
        m.template plane<2>();
        m.template plane<3>();
    }
}

// Can the slices launch run this lattice?  (The march's 32-bit offsets and
// its window width.)
bool slices_ok(int nx, int ny, size_t plane_elems) {
    return nx % 2 == 0 && nx >= 64 && ny >= 8 && 6 * (unsigned long long)plane_elems < (1ull << 32);
}

// Launch 1 of the slices step for the plane set PS.
template <typename T, int PS>
cudaError_t slices_launch(const void *in, void *out, const uint32_t *idx3, const void *rec,
                          int nx, int ny, int nz, int pitch, size_t plane_elems, int num_sms,
                          cudaStream_t st) {
    using M = march::March<T, PS, 2, V_NONE, false>;
    const size_t smem = sizeof(typename M::Slot) * march::NSLOT * march::WARPS;
    auto k1 = k3_slices<T, PS>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    static int per_sm = 1;
    std::call_once(once, [&] {
        attr = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (attr == cudaSuccess)
            attr = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k1, 32 * march::WARPS,
                                                                 smem);
        if (per_sm < 1) per_sm = 1;
    });
    if (attr != cudaSuccess) return attr;
    // launch 1: items of 64-column windows (56 stored) x row segments x slices,
    // about two per resident warp slot
    const int n_wx = (nx + 55) / 56;
    const long long resident = (long long)per_sm * march::WARPS * num_sms;
    long long n_wy = 2 * resident / ((long long)n_wx * nz);
    if (n_wy < 1) n_wy = 1;
    int seg_h = int((ny + n_wy - 1) / n_wy);
    seg_h = seg_h < 32 ? 32 : (seg_h + 3) / 4 * 4;
    n_wy = (ny + seg_h - 1) / seg_h;
    const long long n_items = (long long)n_wx * n_wy * nz;
    const long long blocks = (n_items + march::WARPS - 1) / march::WARPS;
    k1<<<unsigned(blocks), 32 * march::WARPS, smem, st>>>(
        static_cast<const T *>(in), static_cast<T *>(out), idx3,
        static_cast<const MedRec<T> *>(rec), nx, ny, pitch, plane_elems, seg_h, n_wx, int(n_wy),
        n_items);
    return cudaGetLastError();
}

// Kernels one slices step launches: double-single runs launch 1 once per
// triple (a six-plane launch needs 250 registers, two blocks per SM).
template <typename T> constexpr int slices_launches() {
    return std::is_same<T, dsf>::value ? 3 : 2;
}

template <typename T, int VM>
cudaError_t slices_t(const void *in, void *out, const uint32_t *idx3, const void *rec,
                     const void *rv, int nx, int ny, int nz, int pitch, size_t plane_elems,
                     int num_sms, cudaStream_t st) {
    cudaError_t e;
    if constexpr (std::is_same<T, dsf>::value) {
        e = slices_launch<T, P_TE6>(in, out, idx3, rec, nx, ny, nz, pitch, plane_elems, num_sms,
                                    st);
        if (e == cudaSuccess)
            e = slices_launch<T, P_TM6>(in, out, idx3, rec, nx, ny, nz, pitch, plane_elems,
                                        num_sms, st);
    } else {
        e = slices_launch<T, 6>(in, out, idx3, rec, nx, ny, nz, pitch, plane_elems, num_sms, st);
    }
    if (e != cudaSuccess) return e;
    // launch 2: one thread per column, z segments for about two waves of
    // 128-thread blocks (at least 16 planes each)
    const long long cols = (long long)nx * ny;
    const long long cblocks = (cols + 127) / 128;
    int nseg = int((2LL * 8 * num_sms + cblocks - 1) / cblocks);
    if (nseg < 1) nseg = 1;
    int seg = (nz + nseg - 1) / nseg;
    if (seg < 16) seg = 16;
    nseg = (nz + seg - 1) / seg;
    // FP32 loads four planes ahead (3.5% faster than one at 256^3); FP64 is
    // bound by its FMA pipe and loads one ahead; double-single two
    k3_zcol<T, VM, sizeof(T) == 4 ? 4 : (std::is_same<T, dsf>::value ? 2 : 1)><<<dim3(unsigned(cblocks), nseg), 128, 0, st>>>(
        static_cast<const T *>(out), static_cast<T *>(const_cast<void *>(in)), idx3,
        static_cast<const MedRec<T> *>(rec), static_cast<const V3<T> *>(rv), nx, ny, nz, pitch,
        plane_elems, seg);
    return cudaGetLastError();
}

// Records for the register-resident step (kernel 2).  A site whose six
// neighbours carry its own n has zero potential angles, and its record
// depends on n alone: such sites share one record per distinct n through an
// open-addressing table of UNIFORM_SLOTS keys (n's bits; n > 0, so a key is
// never 0, the empty mark), and in a piecewise-uniform medium that is the
// bulk of the lattice, whose records then stay in cache.  Every other site
// gets its own record.  idx3 maps each stored site to its record; rec holds
// the collision coefficient in MedRec form (read by the 2D marching
// machinery; its potential part is unused) and rv the potential
// coefficients.  Index values depend on scheduling, record contents do not.
template <typename T>
__global__ void k3_dedup(const double *__restrict__ n, int nx, int ny, int nz, int pitch,
                         double delta, double vscale, unsigned long long *__restrict__ keys,
                         unsigned *__restrict__ counter, uint32_t *__restrict__ idx3,
                         MedRec<T> *__restrict__ rec, V3<T> *__restrict__ rv,
                         MedRec<dsf> *__restrict__ rec_ds, V3<dsf> *__restrict__ rv_ds) {
    namespace cg = cooperative_groups;
    const size_t N = size_t(nx) * ny * nz;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int x = int(t % nx), y = int((t / nx) % ny), z = int(t / (size_t(nx) * ny));
        const size_t g = at3(x, y, z, ny, pitch);
        const double nn = n[g];
        const double xp = n[at3(wrap(x + 1, nx), y, z, ny, pitch)];
        const double xm = n[at3(wrap(x - 1, nx), y, z, ny, pitch)];
        const double yp = n[at3(x, wrap(y + 1, ny), z, ny, pitch)];
        const double ym = n[at3(x, wrap(y - 1, ny), z, ny, pitch)];
        const double zp = n[at3(x, y, wrap(z + 1, nz), ny, pitch)];
        const double zm = n[at3(x, y, wrap(z - 1, nz), ny, pitch)];
        bool shared = xp == nn && xm == nn && yp == nn && ym == nn && zp == nn && zm == nn;
        bool owner = false;
        uint32_t id = 0;
        if (shared) {
            const unsigned long long key = static_cast<unsigned long long>(__double_as_longlong(nn));
            unsigned h = unsigned(mix64(key)) & (UNIFORM_SLOTS - 1);
            bool placed = false;
            for (int probe = 0; probe < UNIFORM_SLOTS; ++probe) {
                // found with a plain read once placed (no contended atomic)
                if (__ldcg(&keys[h]) == key) {
                    id = h;
                    placed = true;
                    break;
                }
                const unsigned long long prev = atomicCAS(&keys[h], 0ull, key);
                if (prev == 0ull || prev == key) {
                    owner = prev == 0ull;
                    id = h;
                    placed = true;
                    break;
                }
                h = (h + 1) & (UNIFORM_SLOTS - 1);
            }
            shared = placed;  // a full table: fall back to an own record
        }
        if (!shared) {
            cg::coalesced_group grp = cg::coalesced_threads();
            unsigned base = 0;
            if (grp.thread_rank() == 0) base = atomicAdd(counter, grp.size());
            base = grp.shfl(base, 0);
            id = UNIFORM_SLOTS + base + grp.thread_rank();
            owner = true;
        }
        if (owner) {
            // the expressions of k3_medium, so the coefficients are the same
            const double bx = (xp - xm) / (2.0 * delta) / (nn * nn) * delta * delta;
            const double by = (yp - ym) / (2.0 * delta) / (nn * nn) * delta * delta;
            const double bz = (zp - zm) / (2.0 * delta) / (nn * nn) * delta * delta;
            MedRec<T> r{};
            coef_c(delta / (4.0 * nn), r.c);
            rec[id] = r;
            V3<T> v;
            coef_v(vscale * bx, v.gx, v.sx);
            coef_v(vscale * by, v.gy, v.sy);
            coef_v(vscale * bz, v.gz, v.sz);
            rv[id] = v;
            if (rec_ds) {   // QLA_DOUBLE_SINGLE: the same records in word triples
                MedRec<dsf> rd{};
                coef_ds(delta / (4.0 * nn), rd.c);
                rec_ds[id] = rd;
                V3<dsf> vd;
                coef_ds(vscale * bx, vd.x);
                coef_ds(vscale * by, vd.y);
                coef_ds(vscale * bz, vd.z);
                rv_ds[id] = vd;
            }
        }
        idx3[g] = id;
    }
}

// The E_z packet of Sec. V-B, uniform along z: per slice exactly the 2D
// packet (minimum-image xi, eta in the x-y plane, q2 = n E_z, q3 = sin(phi)
// q2, q4 = -cos(phi) q2, the other planes zero).
__device__ __forceinline__ double min_image3(double x, double x0, double L) {
    double d = fmod(x - x0 + 0.5 * L, L);
    if (d < 0.0) d += L;
    return d - 0.5 * L;
}

template <typename T>
__global__ void k3_packet(const double *__restrict__ n, T *__restrict__ q, int nx, int ny, int nz,
                          int pitch, size_t plane_elems, double delta, qla_packet p, double cphi,
                          double sphi) {
    const size_t N = size_t(nx) * ny * nz;
    const double Lx = nx * delta, Ly = ny * delta;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int x = int(t % nx), y = int((t / nx) % ny), z = int(t / (size_t(nx) * ny));
        const size_t g = at3(x, y, z, ny, pitch);
        const double dx = min_image3(x * delta, p.x0, Lx);
        const double dy = min_image3(y * delta, p.y0, Ly);
        const double xi = dx * cphi + dy * sphi;
        const double eta = -dx * sphi + dy * cphi;
        double ez = p.amplitude * exp(-(xi * xi) / (p.width * p.width)) * cos(p.k0 * xi);
        if (p.transverse_width > 0.0)
            ez *= exp(-(eta * eta) / (p.transverse_width * p.transverse_width));
        const double q2 = n[g] * ez;
        q[2 * plane_elems + g] = T(q2);
        q[3 * plane_elems + g] = T(sphi * q2);
        q[4 * plane_elems + g] = T(-cphi * q2);
    }
}

// Gauss laws in 3D (Eqs. 3.1, 3.2; the monitors the paper keeps in its 3D
// runs): div B = d_x q3 + d_y q4 + d_z q5, div D = d_x (n q0) + d_y (n q1)
// + d_z (n q2), centred periodic differences, FP64 sums per block of the
// squares and of the squared diagonal derivatives, and the maxima.
__device__ __forceinline__ double bsum3(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
    if (threadIdx.x < 32)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    return v;
}
__device__ __forceinline__ double bmax3(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
    if (threadIdx.x < 32)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    return v;
}

template <typename T>
__global__ void __launch_bounds__(256)
k3_div(const T *__restrict__ q, const double *__restrict__ n, int nx, int ny, int nz, int pitch,
       size_t plane_elems, double h, double *__restrict__ partials) {
    __shared__ double sh[8];
    const size_t N = size_t(nx) * ny * nz;
    double sb = 0.0, gb = 0.0, sd = 0.0, gd = 0.0, mb = 0.0, md = 0.0;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int x = int(t % nx), y = int((t / nx) % ny), z = int(t / (size_t(nx) * ny));
        const size_t xp = at3(wrap(x + 1, nx), y, z, ny, pitch), xm = at3(wrap(x - 1, nx), y, z, ny, pitch);
        const size_t yp = at3(x, wrap(y + 1, ny), z, ny, pitch), ym = at3(x, wrap(y - 1, ny), z, ny, pitch);
        const size_t zp = at3(x, y, wrap(z + 1, nz), ny, pitch), zm = at3(x, y, wrap(z - 1, nz), ny, pitch);
        const double bx = h * (double(q[3 * plane_elems + xp]) - double(q[3 * plane_elems + xm]));
        const double by = h * (double(q[4 * plane_elems + yp]) - double(q[4 * plane_elems + ym]));
        const double bz = h * (double(q[5 * plane_elems + zp]) - double(q[5 * plane_elems + zm]));
        const double dx = h * (n[xp] * double(q[xp]) - n[xm] * double(q[xm]));
        const double dy = h * (n[yp] * double(q[plane_elems + yp]) - n[ym] * double(q[plane_elems + ym]));
        const double dz = h * (n[zp] * double(q[2 * plane_elems + zp]) -
                               n[zm] * double(q[2 * plane_elems + zm]));
        const double db = bx + by + bz, dd = dx + dy + dz;
        sb = fma(db, db, sb);
        gb = fma(bx, bx, fma(by, by, fma(bz, bz, gb)));
        sd = fma(dd, dd, sd);
        gd = fma(dx, dx, fma(dy, dy, fma(dz, dz, gd)));
        mb = fmax(mb, fabs(db));
        md = fmax(md, fabs(dd));
    }
    const double r0 = bsum3(sb, sh), r1 = bsum3(gb, sh), r2 = bsum3(sd, sh), r3 = bsum3(gd, sh);
    const double r4 = bmax3(mb, sh), r5 = bmax3(md, sh);
    if (threadIdx.x == 0) {
        double *p = partials + size_t(blockIdx.x) * 6;
        p[0] = r0; p[1] = r1; p[2] = r2; p[3] = r3; p[4] = r4; p[5] = r5;
    }
}

__global__ void __launch_bounds__(256)
k3_div_final(const double *__restrict__ partials, int count, double *__restrict__ out) {
    __shared__ double sh[8];
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < count; t += blockDim.x)
        for (int k = 0; k < 6; ++k) {
            const double p = partials[size_t(t) * 6 + k];
            v[k] = k < 4 ? v[k] + p : fmax(v[k], p);
        }
    double r[6];
    for (int k = 0; k < 6; ++k) r[k] = k < 4 ? bsum3(v[k], sh) : bmax3(v[k], sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) out[k] = r[k];
}

}  // namespace
}  // namespace qla

using namespace qla;

struct qla3_ctx {
    int nx = 0, ny = 0, nz = 0, pitch = 0, prec = 0, vmode = V_ROTATION, device = 0;
    double delta = 1.0;
    size_t plane_elems = 0;
    cudaStream_t stream = nullptr;
    char *ws = nullptr;
    bool owns_ws = false;
    void *state[2] = {nullptr, nullptr};
    int cur = 0;
    double *n = nullptr, *staging = nullptr, *partials = nullptr, *result = nullptr;
    void *kc = nullptr, *kv = nullptr;
    // kernel 2: per-site record index, records (shared where uniform)
    uint32_t *idx3 = nullptr;
    void *rec = nullptr, *rv = nullptr;
    // QLA_DOUBLE_SINGLE: double-single records, indexed like rec and rv
    bool ds = false;
    void *rec_ds = nullptr, *rv_ds = nullptr;
    unsigned long long *keys = nullptr;
    unsigned *counter = nullptr;
    int eblocks = 1;
    int num_sms = 1;
    int kernel = 0;   // 0: automatic, 1: fused march along z, 2: slices + column
                      // pipeline, 3: one pass per axis
    bool has_medium = false, has_state = false;
    long long launches = 0;
    qla_status sticky = QLA_OK;
    std::string err;
};

namespace {

struct Layout3 {
    size_t state[2], n, staging, kc, kv, idx3, rec, rv, keys, counter, partials, result, total,
        plane_elems, rec_ds, rv_ds;
    int pitch, eblocks;
};

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

bool dims_ok(int nx, int ny, int nz) {
    return nx >= 1 && ny >= 1 && nz >= 1 && ny <= 65535 && nz <= 65535 &&
           size_t(nx) * ny * nz <= (size_t(1) << 31);
}

Layout3 layout3(int nx, int ny, int nz, int prec, bool ds) {
    Layout3 L{};
    const size_t elt = prec == QLA_FP64 ? 8 : 4;
    L.pitch = (nx + 31) / 32 * 32;
    L.plane_elems = size_t(nz) * ny * L.pitch;
    const size_t sites = size_t(nx) * ny * nz;
    size_t nb = (sites + 2047) / 2048;
    nb = nb > 4096 ? 4096 : (nb < 1 ? 1 : nb);
    L.eblocks = int(nb);
    const size_t kcb = prec == QLA_FP64 ? sizeof(double2) : sizeof(float4);
    const size_t kvb = prec == QLA_FP64 ? sizeof(V3<double>) : sizeof(V3<float>);
    size_t off = 0;
    L.state[0] = off; off += al256(L.plane_elems * elt * 6);
    L.state[1] = off; off += al256(L.plane_elems * elt * 6);
    L.n = off;        off += al256(L.plane_elems * 8);
    L.staging = off;  off += al256(sites * 8);
    L.kc = off;       off += al256(L.plane_elems * kcb);
    L.kv = off;       off += al256(L.plane_elems * kvb);
    const size_t recb = prec == QLA_FP64 ? sizeof(MedRec<double>) : sizeof(MedRec<float>);
    const size_t nrec = UNIFORM_SLOTS + sites;
    L.idx3 = off;     off += al256(L.plane_elems * 4);
    L.rec = off;      off += al256(nrec * recb);
    L.rv = off;       off += al256(nrec * kvb);
    L.keys = off;     off += al256(UNIFORM_SLOTS * 8);
    L.counter = off;  off += al256(4);
    L.partials = off; off += al256(nb * 8 * 6);   // six terms per block (divergence)
    L.result = off;   off += al256(8 * 6);
    L.rec_ds = L.rv_ds = 0;
    if (ds) {
        L.rec_ds = off; off += al256(nrec * sizeof(MedRec<dsf>));
        L.rv_ds = off;  off += al256(nrec * sizeof(V3<dsf>));
    }
    L.total = off;
    return L;
}

qla_status fail3(qla3_ctx *c, qla_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
    if (s == QLA_ECUDA) c->sticky = s;
    return s;
}

#define CUDA3(c, call, what)                                                                \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail3(c, QLA_ECUDA, "%s: %s", what, cudaGetErrorString(e_));             \
    } while (0)

qla_status usable3(qla3_ctx *c) {
    if (!c) return QLA_EINVAL;
    if (c->sticky != QLA_OK) return c->sticky;
    if (cudaSetDevice(c->device) != cudaSuccess) return fail3(c, QLA_ECUDA, "cannot select device");
    return QLA_OK;
}

template <typename T>
cudaError_t step3_t(qla3_ctx *c) {
    const int nx = c->nx, ny = c->ny, nz = c->nz, pitch = c->pitch;
    const size_t pe = c->plane_elems;
    void *a = c->state[c->cur], *b = c->state[c->cur ^ 1];
    // automatic choice: the slices launch for FP32 (1.8x the passes at
    // 256^3), the passes for FP64 (FP64-pipe bound, where the slices'
    // window halo costs more than their fewer memory passes save)
    const int kernel = c->kernel != 0 ? c->kernel : (sizeof(T) == 4 ? 2 : 3);
    if (kernel == 2 && slices_ok(nx, ny, pe)) {
        // the slices launch writes b; the column launch reads b, writes a
        cudaError_t e = c->vmode == V_ROTATION
            ? slices_t<T, V_ROTATION>(a, b, c->idx3, c->rec, c->rv, nx, ny, nz, pitch, pe,
                                      c->num_sms, c->stream)
            : slices_t<T, V_NONE>(a, b, c->idx3, c->rec, c->rv, nx, ny, nz, pitch, pe,
                                  c->num_sms, c->stream);
        c->launches += 2;
        return e;   // the result is back in state[cur]
    }
    if (kernel == 1) {
        cudaError_t e = c->vmode == V_ROTATION
            ? march3_t<T, V_ROTATION>(a, b, c->kc, c->kv, nx, ny, nz, pitch, pe, c->num_sms, c->stream)
            : march3_t<T, V_NONE>(a, b, c->kc, c->kv, nx, ny, nz, pitch, pe, c->num_sms, c->stream);
        c->launches += 1;
        c->cur ^= 1;
        return e;
    }
    cudaError_t e = pass_t<T, 0, false, V_NONE>(a, b, c->kc, c->kv, nx, ny, nz, pitch, pe, c->stream);
    if (e != cudaSuccess) return e;
    e = pass_t<T, 1, false, V_NONE>(b, a, c->kc, c->kv, nx, ny, nz, pitch, pe, c->stream);
    if (e != cudaSuccess) return e;
    e = c->vmode == V_ROTATION
            ? pass_t<T, 2, true, V_ROTATION>(a, b, c->kc, c->kv, nx, ny, nz, pitch, pe, c->stream)
            : pass_t<T, 2, true, V_NONE>(a, b, c->kc, c->kv, nx, ny, nz, pitch, pe, c->stream);
    c->launches += 3;
    c->cur ^= 1;
    return e;
}

}  // namespace

extern "C" {

size_t qla3_workspace_bytes(int nx, int ny, int nz, int precision, unsigned flags) {
    if (!dims_ok(nx, ny, nz) || (precision != QLA_FP64 && precision != QLA_FP32)) return 0;
    if (flags & ~(unsigned)(QLA_POTENTIAL_NONE | QLA_DOUBLE_SINGLE)) return 0;
    const bool ds = (flags & QLA_DOUBLE_SINGLE) != 0;
    if (ds && (precision != QLA_FP64 ||
               !slices_ok(nx, ny, size_t(nz) * ny * size_t((nx + 31) / 32 * 32))))
        return 0;
    return layout3(nx, ny, nz, precision, ds).total;
}

qla_status qla3_init(qla3_ctx **out, int nx, int ny, int nz, double delta, int precision,
                     unsigned flags, void *cuda_stream, void *workspace, size_t workspace_bytes) {
    if (!out) return QLA_EINVAL;
    *out = nullptr;
    const size_t need = qla3_workspace_bytes(nx, ny, nz, precision, flags);
    if (need == 0 || !(delta > 0.0) || !std::isfinite(delta)) return QLA_EINVAL;
    if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255)) return QLA_EINVAL;
    if (workspace && workspace_bytes < need) return QLA_ENOMEM;
    qla3_ctx *c = new (std::nothrow) qla3_ctx();
    if (!c) return QLA_ENOMEM;
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->delta = delta;
    c->prec = precision;
    c->vmode = (flags & QLA_POTENTIAL_NONE) ? V_NONE : V_ROTATION;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return QLA_ECUDA; }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (c->num_sms < 1) c->num_sms = 1;
    c->ds = (flags & QLA_DOUBLE_SINGLE) != 0;
    const Layout3 L = layout3(nx, ny, nz, precision, c->ds);
    if (workspace) {
        c->ws = static_cast<char *>(workspace);
    } else {
        void *p = nullptr;
        if (cudaMalloc(&p, L.total) != cudaSuccess) { cudaGetLastError(); delete c; return QLA_ENOMEM; }
        c->ws = static_cast<char *>(p);
        c->owns_ws = true;
    }
    c->pitch = L.pitch;
    c->plane_elems = L.plane_elems;
    c->state[0] = c->ws + L.state[0];
    c->state[1] = c->ws + L.state[1];
    c->n = reinterpret_cast<double *>(c->ws + L.n);
    c->staging = reinterpret_cast<double *>(c->ws + L.staging);
    c->kc = c->ws + L.kc;
    c->kv = c->ws + L.kv;
    c->idx3 = reinterpret_cast<uint32_t *>(c->ws + L.idx3);
    c->rec = c->ws + L.rec;
    c->rv = c->ws + L.rv;
    if (c->ds) {
        c->rec_ds = c->ws + L.rec_ds;
        c->rv_ds = c->ws + L.rv_ds;
    }
    c->keys = reinterpret_cast<unsigned long long *>(c->ws + L.keys);
    c->counter = reinterpret_cast<unsigned *>(c->ws + L.counter);
    c->partials = reinterpret_cast<double *>(c->ws + L.partials);
    c->result = reinterpret_cast<double *>(c->ws + L.result);
    c->eblocks = L.eblocks;
    // both state buffers start at zero (pad columns included)
    if (cudaMemsetAsync(c->ws, 0, L.n, c->stream) != cudaSuccess) {
        cudaGetLastError();
        if (c->owns_ws) cudaFree(c->ws);
        delete c;
        return QLA_ECUDA;
    }
    *out = c;
    return QLA_OK;
}

qla_status qla3_set_medium(qla3_ctx *c, const double *n_host) {
    qla_status s = usable3(c);
    if (s != QLA_OK) return s;
    if (!n_host) return fail3(c, QLA_EINVAL, "qla3_set_medium: null n");
    const size_t N = size_t(c->nx) * c->ny * c->nz;
    for (size_t k = 0; k < N; ++k)
        if (!(n_host[k] > 0.0) || !std::isfinite(n_host[k]))
            return fail3(c, QLA_EINVAL, "qla3_set_medium: n[%zu] = %g is not finite and > 0", k,
                         n_host[k]);
    const int rows = c->ny * c->nz;
    CUDA3(c, cudaMemcpyAsync(c->staging, n_host, N * 8, cudaMemcpyHostToDevice, c->stream),
          "qla3_set_medium: copy");
    CUDA3(c, raw_pitch_copy(c->staging, c->n, c->nx, rows, c->pitch, c->stream),
          "qla3_set_medium: place");
    const double vscale = 0.5;   // rotation reading: V rotates by beta / 2
    const int blocks = int(std::min<size_t>((N + 255) / 256, size_t(65535) * 16));
    if (c->prec == QLA_FP64)
        k3_medium<double><<<blocks, 256, 0, c->stream>>>(
            c->n, c->nx, c->ny, c->nz, c->pitch, c->delta, vscale,
            static_cast<double2 *>(c->kc), static_cast<V3<double> *>(c->kv));
    else
        k3_medium<float><<<blocks, 256, 0, c->stream>>>(
            c->n, c->nx, c->ny, c->nz, c->pitch, c->delta, vscale,
            static_cast<float4 *>(c->kc), static_cast<V3<float> *>(c->kv));
    CUDA3(c, cudaGetLastError(), "qla3_set_medium: kernel");
    CUDA3(c, cudaMemsetAsync(c->keys, 0, UNIFORM_SLOTS * 8, c->stream), "qla3_set_medium: clear");
    CUDA3(c, cudaMemsetAsync(c->counter, 0, 4, c->stream), "qla3_set_medium: clear");
    if (c->prec == QLA_FP64)
        k3_dedup<double><<<blocks, 256, 0, c->stream>>>(
            c->n, c->nx, c->ny, c->nz, c->pitch, c->delta, vscale, c->keys, c->counter, c->idx3,
            static_cast<MedRec<double> *>(c->rec), static_cast<V3<double> *>(c->rv),
            static_cast<MedRec<dsf> *>(c->rec_ds), static_cast<V3<dsf> *>(c->rv_ds));
    else
        k3_dedup<float><<<blocks, 256, 0, c->stream>>>(
            c->n, c->nx, c->ny, c->nz, c->pitch, c->delta, vscale, c->keys, c->counter, c->idx3,
            static_cast<MedRec<float> *>(c->rec), static_cast<V3<float> *>(c->rv), nullptr,
            nullptr);
    CUDA3(c, cudaGetLastError(), "qla3_set_medium: records");
    c->launches += 3;
    CUDA3(c, cudaStreamSynchronize(c->stream), "qla3_set_medium: sync");
    c->has_medium = true;
    return QLA_OK;
}

qla_status qla3_set_state(qla3_ctx *c, const double *q_host) {
    qla_status s = usable3(c);
    if (s != QLA_OK) return s;
    if (!q_host) return fail3(c, QLA_EINVAL, "qla3_set_state: null state");
    const size_t N = size_t(c->nx) * c->ny * c->nz;
    for (size_t k = 0; k < 6 * N; ++k)
        if (!std::isfinite(q_host[k]))
            return fail3(c, QLA_EINVAL, "qla3_set_state: non-finite value at %zu", k);
    const size_t elt = c->prec == QLA_FP64 ? 8 : 4;
    for (int comp = 0; comp < 6; ++comp) {
        CUDA3(c, cudaMemcpyAsync(c->staging, q_host + size_t(comp) * N, N * 8,
                                 cudaMemcpyHostToDevice, c->stream), "qla3_set_state: copy");
        CUDA3(c, raw_from_f64(c->prec, c->staging,
                              static_cast<char *>(c->state[c->cur]) + comp * c->plane_elems * elt,
                              c->nx, c->ny * c->nz, c->pitch, c->stream),
              "qla3_set_state: convert");
        c->launches++;
    }
    // the staging plane is reused per component and the host buffer may
    // change after return
    CUDA3(c, cudaStreamSynchronize(c->stream), "qla3_set_state: sync");
    c->has_state = true;
    return QLA_OK;
}

qla_status qla3_get_state(qla3_ctx *c, double *q_host) {
    qla_status s = usable3(c);
    if (s != QLA_OK) return s;
    if (!q_host) return fail3(c, QLA_EINVAL, "qla3_get_state: null output");
    if (!c->has_state) return fail3(c, QLA_ESTATE, "qla3_get_state: no state");
    const size_t N = size_t(c->nx) * c->ny * c->nz;
    for (int comp = 0; comp < 6; ++comp) {
        CUDA3(c, raw_to_f64(c->prec, c->state[c->cur], c->plane_elems, comp, c->staging, c->nx,
                            c->ny * c->nz, c->pitch, c->stream), "qla3_get_state: convert");
        c->launches++;
        CUDA3(c, cudaMemcpyAsync(q_host + size_t(comp) * N, c->staging, N * 8,
                                 cudaMemcpyDeviceToHost, c->stream), "qla3_get_state: copy");
        CUDA3(c, cudaStreamSynchronize(c->stream), "qla3_get_state: sync");
    }
    return QLA_OK;
}

qla_status qla3_step(qla3_ctx *c, long long n_steps) {
    qla_status s = usable3(c);
    if (s != QLA_OK) return s;
    if (n_steps < 0) return fail3(c, QLA_EINVAL, "qla3_step: n_steps < 0");
    if (n_steps == 0) return QLA_OK;
    if (!c->has_medium || !c->has_state)
        return fail3(c, QLA_ESTATE, "qla3_step: set a medium and a state first");
    if (c->ds) {
        // word pairs in place, n double-single steps (slices + column
        // pipeline; the result returns to state[cur]), back to FP64
        const size_t n = 6 * c->plane_elems;
        CUDA3(c, raw_to_ds(c->state[c->cur], n, c->stream), "qla3_step: to double-single");
        void *a = c->state[c->cur], *b = c->state[c->cur ^ 1];
        for (long long k = 0; k < n_steps; ++k) {
            const cudaError_t e =
                c->vmode == V_ROTATION
                    ? slices_t<dsf, V_ROTATION>(a, b, c->idx3, c->rec_ds, c->rv_ds, c->nx, c->ny,
                                                c->nz, c->pitch, c->plane_elems, c->num_sms,
                                                c->stream)
                    : slices_t<dsf, V_NONE>(a, b, c->idx3, c->rec_ds, c->rv_ds, c->nx, c->ny,
                                            c->nz, c->pitch, c->plane_elems, c->num_sms,
                                            c->stream);
            CUDA3(c, e, "qla3_step: kernel");
            c->launches += slices_launches<dsf>();
        }
        CUDA3(c, raw_from_ds(c->state[c->cur], n, c->stream), "qla3_step: from double-single");
        c->launches += 2;
        return QLA_OK;
    }
    for (long long k = 0; k < n_steps; ++k)
        CUDA3(c, c->prec == QLA_FP64 ? step3_t<double>(c) : step3_t<float>(c), "qla3_step: kernel");
    return QLA_OK;
}

qla_status qla3_energy(qla3_ctx *c, double *out) {
    qla_status s = usable3(c);
    if (s != QLA_OK) return s;
    if (!out) return fail3(c, QLA_EINVAL, "qla3_energy: null output");
    if (!c->has_state) return fail3(c, QLA_ESTATE, "qla3_energy: no state");
    CUDA3(c, raw_energy(c->prec, c->state[c->cur], c->plane_elems, c->nx, c->ny * c->nz, c->pitch,
                        c->partials, c->eblocks, c->result, c->stream), "qla3_energy: kernel");
    c->launches += 2;
    CUDA3(c, cudaMemcpyAsync(out, c->result, 8, cudaMemcpyDeviceToHost, c->stream),
          "qla3_energy: copy");
    CUDA3(c, cudaStreamSynchronize(c->stream), "qla3_energy: sync");
    if (!std::isfinite(*out)) return fail3(c, QLA_ENONFINITE, "qla3_energy: energy is %g", *out);
    return QLA_OK;
}

qla_status qla3_set_step_kernel(qla3_ctx *c, int kernel) {
    qla_status s = usable3(c);
    if (s != QLA_OK) return s;
    if (kernel < 0 || kernel > 3)
        return fail3(c, QLA_EINVAL, "qla3_set_step_kernel: kernel must be 0..3, got %d", kernel);
    c->kernel = kernel;
    return QLA_OK;
}

qla_status qla3_set_packet(qla3_ctx *c, const qla_packet *p) {
    qla_status s = usable3(c);
    if (s != QLA_OK) return s;
    if (!p) return fail3(c, QLA_EINVAL, "qla3_set_packet: null packet");
    const double v[7] = {p->x0, p->y0, p->angle, p->k0, p->width, p->transverse_width,
                         p->amplitude};
    for (double x : v)
        if (!std::isfinite(x)) return fail3(c, QLA_EINVAL, "qla3_set_packet: non-finite field");
    if (!(p->width > 0.0) || p->transverse_width < 0.0)
        return fail3(c, QLA_EINVAL, "qla3_set_packet: width must be > 0, transverse_width >= 0");
    if (!c->has_medium) return fail3(c, QLA_ESTATE, "qla3_set_packet: set the medium first");
    const size_t elt = c->prec == QLA_FP64 ? 8 : 4;
    CUDA3(c, cudaMemsetAsync(c->state[c->cur], 0, c->plane_elems * elt * 6, c->stream),
          "qla3_set_packet: clear");
    const size_t N = size_t(c->nx) * c->ny * c->nz;
    const int blocks = int(std::min<size_t>((N + 255) / 256, size_t(65535) * 16));
    const double cphi = cos(p->angle), sphi = sin(p->angle);
    if (c->prec == QLA_FP64)
        k3_packet<double><<<blocks, 256, 0, c->stream>>>(
            c->n, static_cast<double *>(c->state[c->cur]), c->nx, c->ny, c->nz, c->pitch,
            c->plane_elems, c->delta, *p, cphi, sphi);
    else
        k3_packet<float><<<blocks, 256, 0, c->stream>>>(
            c->n, static_cast<float *>(c->state[c->cur]), c->nx, c->ny, c->nz, c->pitch,
            c->plane_elems, c->delta, *p, cphi, sphi);
    CUDA3(c, cudaGetLastError(), "qla3_set_packet: kernel");
    c->launches++;
    c->has_state = true;
    return QLA_OK;
}

qla_status qla3_divergence(qla3_ctx *c, double *out) {
    qla_status s = usable3(c);
    if (s != QLA_OK) return s;
    if (!out) return fail3(c, QLA_EINVAL, "qla3_divergence: null output");
    if (!c->has_state || !c->has_medium)
        return fail3(c, QLA_ESTATE, "qla3_divergence: needs medium and state");
    const double h = 0.5 / c->delta;
    if (c->prec == QLA_FP64)
        k3_div<double><<<c->eblocks, 256, 0, c->stream>>>(
            static_cast<const double *>(c->state[c->cur]), c->n, c->nx, c->ny, c->nz, c->pitch,
            c->plane_elems, h, c->partials);
    else
        k3_div<float><<<c->eblocks, 256, 0, c->stream>>>(
            static_cast<const float *>(c->state[c->cur]), c->n, c->nx, c->ny, c->nz, c->pitch,
            c->plane_elems, h, c->partials);
    CUDA3(c, cudaGetLastError(), "qla3_divergence: kernel");
    k3_div_final<<<1, 256, 0, c->stream>>>(c->partials, c->eblocks, c->result);
    CUDA3(c, cudaGetLastError(), "qla3_divergence: final");
    c->launches += 2;
    CUDA3(c, cudaMemcpyAsync(out, c->result, 6 * 8, cudaMemcpyDeviceToHost, c->stream),
          "qla3_divergence: copy");
    CUDA3(c, cudaStreamSynchronize(c->stream), "qla3_divergence: sync");
    for (int k = 0; k < 6; ++k)
        if (!std::isfinite(out[k]))
            return fail3(c, QLA_ENONFINITE, "qla3_divergence: term %d is %g", k, out[k]);
    return QLA_OK;
}

long long qla3_launch_count(const qla3_ctx *c) { return c ? c->launches : 0; }

const char *qla3_last_error(const qla3_ctx *c) { return c ? c->err.c_str() : "null context"; }

void qla3_destroy(qla3_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->owns_ws) cudaFree(c->ws);
    delete c;
}

}  // extern "C"
