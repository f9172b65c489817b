// Generic QLA step kernel: one step of Eq. 2e14 per launch, any lattice size,
// FP64 or FP32, six planes or the E_z triple, every potential reading.
//
// A CTA owns a TX x TY tile of outputs.  U_x and U_y each reach four cells
// along their axis (four of their eight layers pair neighbouring sites), so
// the CTA stages the tile plus a 4-cell periodic halo of every live plane
// and of the collision coefficients in shared memory.  U_x is applied to
// every staged row, U_y to the tile's columns, as eight layers of disjoint
// 2x2 rotations each (see layer_of in qla_internal.h); bonds that would
// leave the staged region are skipped, which only corrupts halo cells that
// no output depends on.  The previous step's V_x, V_y (when pending) are
// applied to every staged site on load; the buffer written holds U_y U_x Q.
// For a diagonal index tensor (six planes) the kernel stages a coefficient
// per pair class and applies this step's V before storing instead; so it
// does for the LCU form of V (Eqs. 2f1-2f7).
#include <type_traits>

#include "qla_internal.h"

namespace qla {
namespace {

constexpr int HALO = 4;
constexpr int THREADS = 256;

template <typename T> struct TileShape;
template <> struct TileShape<double> { static constexpr int TX = 32, TY = 16; };
template <> struct TileShape<float>  { static constexpr int TX = 32, TY = 32; };

// Staged collision coefficients of a diagonal index tensor: one per pair
// class (see MedRecT).
template <typename T> struct TriC { typename Coef<T>::C c15, c2, c05; };

// The coefficient of pair pk (0: the pair with q5, 1: the pair with q2) of a
// direction: a scalar medium has one for all pairs.
template <bool XDIR, typename C>
__device__ __forceinline__ C coef_of(C k, int) { return k; }
template <bool XDIR, typename T>
__device__ __forceinline__ typename Coef<T>::C coef_of(const TriC<T> &k, int pk) {
    return pk == 1 ? k.c2 : XDIR ? k.c15 : k.c05;
}

// Apply one bond layer to all pairs of one direction at bond site `i` of a
// line whose elements are `stride` apart in shared memory.
template <typename T, int P, bool XDIR, int L, typename SC>
__device__ __forceinline__ void bond(T *s, size_t plane, int idx, int stride, const SC &k) {
    constexpr Layer ly = layer_of(L);
    // collision sign: C_x rotates by +theta, C_y by -theta; adjoint flips
    constexpr int g0 = XDIR ? 1 : -1;
    const T g = T(ly.dag ? -g0 : g0);
#pragma unroll
    for (int pk = 0; pk < 2; ++pk) {
        constexpr int dummy = 0;
        (void)dummy;
        const Pair pr = pair_of(XDIR, pk);
        const int pa = plane_of<P>(pr.a), pb = plane_of<P>(pr.b);
        if (pa < 0 || pb < 0) continue;
        // which element of the pair sits at i + shift
        int ia = idx, ib = idx;
        if (ly.mover == 1) {
            if (pr.a_is_m1) ia += ly.shift * stride; else ib += ly.shift * stride;
        } else if (ly.mover == 2) {
            if (pr.a_is_m1) ib += ly.shift * stride; else ia += ly.shift * stride;
        }
        T a = s[pa * plane + ia], b = s[pb * plane + ib];
        rotate(a, b, coef_of<XDIR>(k, pk), g);
        s[pa * plane + ia] = a;
        s[pb * plane + ib] = b;
    }
}

template <typename T, int P, bool XDIR, int L, int RX, int RY, int TX, typename SC>
__device__ __forceinline__ void layer_pass(T *s, const SC *sc) {
    constexpr Layer ly = layer_of(L);
    constexpr size_t plane = size_t(RX) * RY;
    if constexpr (XDIR) {
        // every staged row, bond sites i with i + shift inside the row
        for (int t = threadIdx.x; t < RX * RY; t += THREADS) {
            const int r = t / RX, i = t - r * RX;
            const int j = i + ly.shift;
            if (j < 0 || j >= RX) continue;
            bond<T, P, true, L>(s, plane, r * RX + i, 1, sc[r * RX + i]);
        }
    } else {
        // the tile's columns, bond sites r with r + shift inside the column
        for (int t = threadIdx.x; t < TX * RY; t += THREADS) {
            const int r = t / TX, i = HALO + (t - r * TX);
            const int j = r + ly.shift;
            if (j < 0 || j >= RY) continue;
            bond<T, P, false, L>(s, plane, r * RX + i, RX, sc[r * RX + i]);
        }
    }
}

template <typename T, int P, bool XDIR, int RX, int RY, int TX, typename SC>
__device__ __forceinline__ void apply_U(T *s, const SC *sc) {
    layer_pass<T, P, XDIR, 0, RX, RY, TX>(s, sc); __syncthreads();
    layer_pass<T, P, XDIR, 1, RX, RY, TX>(s, sc); __syncthreads();
    layer_pass<T, P, XDIR, 2, RX, RY, TX>(s, sc); __syncthreads();
    layer_pass<T, P, XDIR, 3, RX, RY, TX>(s, sc); __syncthreads();
    layer_pass<T, P, XDIR, 4, RX, RY, TX>(s, sc); __syncthreads();
    layer_pass<T, P, XDIR, 5, RX, RY, TX>(s, sc); __syncthreads();
    layer_pass<T, P, XDIR, 6, RX, RY, TX>(s, sc); __syncthreads();
    layer_pass<T, P, XDIR, 7, RX, RY, TX>(s, sc); __syncthreads();
}

// TS: a diagonal index tensor (QLA_ANISOTROPIC, six planes): per-site
// records in ttable, each pair with its own coefficient, and this step's
// potential operator applied to the outputs before they are stored (no
// pending V; VIN is false).
template <typename T, int P, int VM, bool VIN, bool TS>
__global__ void __launch_bounds__(THREADS)
k_step_tile(const T *__restrict__ in, T *__restrict__ out,
            const uint32_t *__restrict__ midx, const MedRec<T> *__restrict__ table,
            const MedRecT<T> *__restrict__ ttable, int nx, int ny, int pitch,
            size_t plane_elems) {
    using SC = typename std::conditional<TS, TriC<T>, typename Coef<T>::C>::type;
    constexpr int TX = TileShape<T>::TX, TY = TileShape<T>::TY;
    constexpr int RX = TX + 2 * HALO, RY = TY + 2 * HALO;
    constexpr size_t plane = size_t(RX) * RY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SC *sc = reinterpret_cast<SC *>(smem_raw);
    T *s = reinterpret_cast<T *>(sc + plane);

    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    for (int t = threadIdx.x; t < RX * RY; t += THREADS) {
        const int r = t / RX, c = t - r * RX;
        const int gx = wrap(x0 - HALO + c, nx), gy = wrap(y0 - HALO + r, ny);
        const size_t g = size_t(gy) * pitch + gx;
        // the pending potential operator of the previous step first
        T q[6];
        load_site<T, P, VM>(in, plane_elems, g, VIN, midx, table, q);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int p = plane_of<P>(k);
            if (p >= 0) s[p * plane + t] = q[k];
        }
        if constexpr (TS) {
            const MedRecT<T> &r = ttable[g];
            sc[t] = SC{r.c15, r.c2, r.c05};
        } else {
            sc[t] = table[midx[g]].c;
        }
    }
    __syncthreads();
    apply_U<T, P, true, RX, RY, TX>(s, sc);    // U_x (Eq. 2e6)
    apply_U<T, P, false, RX, RY, TX>(s, sc);   // U_y (Eq. 2e9)

    for (int t = threadIdx.x; t < TX * TY; t += THREADS) {
        const int r = t / TX, c = t - r * TX;
        const int gx = x0 + c, gy = y0 + r;
        if (gx >= nx || gy >= ny) continue;
        const int st = (r + HALO) * RX + c + HALO;
        T q[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int p = plane_of<P>(k);
            q[k] = p >= 0 ? s[p * plane + st] : T(0);
        }
        const size_t g = size_t(gy) * pitch + gx;
        if constexpr (TS) {
            const MedRecT<T> &r = ttable[g];
            apply_potential_tensor<T, P, VM>(q, r.vz, r.vt);   // V_y V_x (Eq. 2e14)
        } else if constexpr (VM == V_LCU) {
            apply_potential<T, P, VM>(q, table[midx[g]].v);     // Eqs. 2f1-2f7
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int p = plane_of<P>(k);
            if (p >= 0) out[p * plane_elems + g] = q[k];
        }
    }
}

template <typename T, int P, int VM, bool VIN, bool TS = false>
cudaError_t launch_tile_t(qla_ctx *c, const void *in, void *out) {
    using SC = typename std::conditional<TS, TriC<T>, typename Coef<T>::C>::type;
    constexpr int TX = TileShape<T>::TX, TY = TileShape<T>::TY;
    constexpr int RX = TX + 2 * HALO, RY = TY + 2 * HALO;
    const size_t smem = size_t(RX) * RY * (sizeof(SC) + P * sizeof(T));
    auto kern = k_step_tile<T, P, VM, VIN, TS>;
    // per instantiation, per process; set once (thread-safe)
    static const cudaError_t attr =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (attr != cudaSuccess) return attr;
    dim3 grid((c->nx + TX - 1) / TX, (c->ny + TY - 1) / TY);
    kern<<<grid, THREADS, smem, c->stream>>>(
        static_cast<const T *>(in), static_cast<T *>(out),
        c->midx, static_cast<const MedRec<T> *>(c->table),
        static_cast<const MedRecT<T> *>(c->ttable), c->nx, c->ny, c->pitch, c->plane_elems);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tensor_vm(qla_ctx *c, const void *in, void *out) {
    switch (c->vmode) {
    case V_ROTATION: return launch_tile_t<T, 6, V_ROTATION, false, true>(c, in, out);
    case V_LITERAL:  return launch_tile_t<T, 6, V_LITERAL, false, true>(c, in, out);
    case V_LCU:      return launch_tile_t<T, 6, V_LCU, false, true>(c, in, out);
    default:         return launch_tile_t<T, 6, V_NONE, false, true>(c, in, out);
    }
}

template <typename T, int P>
cudaError_t launch_tile_vm(qla_ctx *c, const void *in, void *out, bool vin) {
    switch (c->vmode) {
    case V_ROTATION:
        return vin ? launch_tile_t<T, P, V_ROTATION, true>(c, in, out)
                   : launch_tile_t<T, P, V_ROTATION, false>(c, in, out);
    case V_LITERAL:
        return vin ? launch_tile_t<T, P, V_LITERAL, true>(c, in, out)
                   : launch_tile_t<T, P, V_LITERAL, false>(c, in, out);
    case V_LCU: return launch_tile_t<T, P, V_LCU, false>(c, in, out);   // V applied at the end
    default: return launch_tile_t<T, P, V_NONE, false>(c, in, out);
    }
}

}  // namespace

cudaError_t launch_step_tensor(qla_ctx *c, const void *in, void *out) {
    return c->prec == QLA_FP64 ? launch_tensor_vm<double>(c, in, out)
                               : launch_tensor_vm<float>(c, in, out);
}

cudaError_t launch_step_tile(qla_ctx *c, const void *in, void *out, bool vin) {
    if (c->prec == QLA_FP64)
        return c->P == 6 ? launch_tile_vm<double, 6>(c, in, out, vin)
                         : launch_tile_vm<double, 3>(c, in, out, vin);
    return c->P == 6 ? launch_tile_vm<float, 6>(c, in, out, vin)
                     : launch_tile_vm<float, 3>(c, in, out, vin);
}

}  // namespace qla
