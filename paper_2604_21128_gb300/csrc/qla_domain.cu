// Domain decomposition (Sec. V-A: the lattice split into processor domains
// that trade boundary points after each step).  A sub-domain is an ordinary
// context on its block of the lattice plus a halo of ghost cells on every
// side; these calls move rectangles of its stored state in and out of
// contiguous device buffers (what the halo exchange sends), sum the energy
// of a rectangle (its interior, for the global FP64 sum), and place the
// Gaussian packet of Sec. V-B on a context that is a window of a larger
// periodic lattice.
#include <cmath>

#include "qla_internal.h"

namespace qla {
namespace {

constexpr int DOM_THREADS = 256;

inline int dom_grid(size_t n) {
    const size_t b = (n + DOM_THREADS - 1) / DOM_THREADS;
    return int(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// dst[p][j][i] = q[p][j0 + j][i0 + i] for every stored plane p, 0 <= j < h,
// 0 <= i < w (TO_BOX); the other way round otherwise.
template <typename T, bool TO_BOX>
__global__ void __launch_bounds__(DOM_THREADS)
k_box_copy(T *__restrict__ q, size_t plane_elems, int pitch, int planes, int i0, int j0, int w,
           int h, T *__restrict__ box) {
    const size_t per_plane = size_t(w) * h, n = per_plane * planes;
    for (size_t t = blockIdx.x * size_t(DOM_THREADS) + threadIdx.x; t < n;
         t += size_t(gridDim.x) * DOM_THREADS) {
        const size_t p = t / per_plane, r = t - p * per_plane;
        const int j = int(r / w), i = int(r - size_t(j) * w);
        const size_t g = p * plane_elems + size_t(j0 + j) * pitch + (i0 + i);
        if (TO_BOX) box[t] = q[g];
        else q[g] = box[t];
    }
}

__device__ double dom_block_sum(double v) {
    __shared__ double part[DOM_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) part[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = lane < DOM_THREADS / 32 ? part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// Sum of q^2 (Eq. A13) over the sites of a rectangle, with the pending
// potential step applied as every read-out does; fixed order per block.
template <typename T, int P, int VM>
__global__ void __launch_bounds__(DOM_THREADS)
k_energy_box(const T *__restrict__ q, size_t plane_elems, int pitch, int i0, int j0, int w, int h,
             bool vin, const uint32_t *__restrict__ midx, const MedRec<T> *__restrict__ table,
             double *__restrict__ partials) {
    const size_t n = size_t(w) * h;
    double acc = 0.0;
    for (size_t t = blockIdx.x * size_t(DOM_THREADS) + threadIdx.x; t < n;
         t += size_t(gridDim.x) * DOM_THREADS) {
        const int j = int(t / w), i = int(t - size_t(j) * w);
        const size_t g = size_t(j0 + j) * pitch + (i0 + i);
        T s[6];
        load_site<T, P, VM>(q, plane_elems, g, vin, midx, table, s);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (plane_of<P>(c) < 0) continue;
            const double v = double(s[c]);
            acc = fma(v, v, acc);
        }
    }
    acc = dom_block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(DOM_THREADS)
k_energy_box_final(const double *__restrict__ partials, int count, double *__restrict__ out) {
    double acc = 0.0;
    for (int t = threadIdx.x; t < count; t += DOM_THREADS) acc += partials[t];
    acc = dom_block_sum(acc);
    if (threadIdx.x == 0) *out = acc;
}

template <typename T, int P>
cudaError_t energy_box_p(qla_ctx *c, int i0, int j0, int w, int h) {
    const T *q = static_cast<const T *>(c->state[c->cur]);
    const MedRec<T> *tb = static_cast<const MedRec<T> *>(c->table);
    const bool vin = c->pending_v;
    const int nb = c->energy_blocks;
    switch (c->vmode) {
    case V_ROTATION:
        k_energy_box<T, P, V_ROTATION><<<nb, DOM_THREADS, 0, c->stream>>>(
            q, c->plane_elems, c->pitch, i0, j0, w, h, vin, c->midx, tb, c->partials);
        break;
    case V_LITERAL:
        k_energy_box<T, P, V_LITERAL><<<nb, DOM_THREADS, 0, c->stream>>>(
            q, c->plane_elems, c->pitch, i0, j0, w, h, vin, c->midx, tb, c->partials);
        break;
    default:
        k_energy_box<T, P, V_NONE><<<nb, DOM_THREADS, 0, c->stream>>>(
            q, c->plane_elems, c->pitch, i0, j0, w, h, false, c->midx, tb, c->partials);
    }
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_energy_box_final<<<1, DOM_THREADS, 0, c->stream>>>(c->partials, nb, c->result);
    c->launches++;
    return cudaGetLastError();
}

// E_z packet on the context's sites taken as the window of a gnx x gny
// periodic lattice whose first site is (i0, j0): the distances are minimum
// images on the large lattice (as qla_set_packet does on the context's own).
__device__ __forceinline__ double dom_min_image(double x, double x0, double L) {
    double d = fmod(x - x0 + 0.5 * L, L);
    if (d < 0.0) d += L;
    return d - 0.5 * L;
}

template <typename T, int P>
__global__ void __launch_bounds__(DOM_THREADS)
k_packet_window(const double *__restrict__ n, T *__restrict__ q, int nx, int ny, int pitch,
                size_t plane_elems, double delta, int i0, int j0, int gnx, int gny, qla_packet p,
                double cphi, double sphi) {
    const size_t N = size_t(nx) * ny;
    const double Lx = gnx * delta, Ly = gny * delta;
    for (size_t t = blockIdx.x * size_t(DOM_THREADS) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * DOM_THREADS) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        const size_t g = size_t(j) * pitch + i;
        int gi = (i0 + i) % gnx, gj = (j0 + j) % gny;
        if (gi < 0) gi += gnx;
        if (gj < 0) gj += gny;
        const double dx = dom_min_image(gi * delta, p.x0, Lx);
        const double dy = dom_min_image(gj * delta, p.y0, Ly);
        const double xi = dx * cphi + dy * sphi;
        const double eta = -dx * sphi + dy * cphi;
        double ez = p.amplitude * exp(-(xi * xi) / (p.width * p.width)) * cos(p.k0 * xi);
        if (p.transverse_width > 0.0)
            ez *= exp(-(eta * eta) / (p.transverse_width * p.transverse_width));
        const double q2 = n[g] * ez;
        const double vals[6] = {0.0, 0.0, q2, sphi * q2, -cphi * q2, 0.0};
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int pl = plane_of<P>(c);
            if (pl >= 0) q[pl * plane_elems + g] = T(vals[c]);
        }
    }
}

template <typename T, int P>
cudaError_t packet_window_p(qla_ctx *c, const qla_packet &p, int i0, int j0, int gnx, int gny) {
    const size_t N = size_t(c->nx) * c->ny;
    k_packet_window<T, P><<<dom_grid(N), DOM_THREADS, 0, c->stream>>>(
        c->n, static_cast<T *>(c->state[c->cur]), c->nx, c->ny, c->pitch, c->plane_elems,
        c->delta, i0, j0, gnx, gny, p, cos(p.angle), sin(p.angle));
    c->launches++;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_box_copy(qla_ctx *c, int i0, int j0, int w, int h, void *box, bool to_box) {
    const size_t n = size_t(w) * h * c->P;
    if (c->prec == QLA_FP64) {
        double *q = static_cast<double *>(c->state[c->cur]);
        if (to_box)
            k_box_copy<double, true><<<dom_grid(n), DOM_THREADS, 0, c->stream>>>(
                q, c->plane_elems, c->pitch, c->P, i0, j0, w, h, static_cast<double *>(box));
        else
            k_box_copy<double, false><<<dom_grid(n), DOM_THREADS, 0, c->stream>>>(
                q, c->plane_elems, c->pitch, c->P, i0, j0, w, h, static_cast<double *>(box));
    } else {
        float *q = static_cast<float *>(c->state[c->cur]);
        if (to_box)
            k_box_copy<float, true><<<dom_grid(n), DOM_THREADS, 0, c->stream>>>(
                q, c->plane_elems, c->pitch, c->P, i0, j0, w, h, static_cast<float *>(box));
        else
            k_box_copy<float, false><<<dom_grid(n), DOM_THREADS, 0, c->stream>>>(
                q, c->plane_elems, c->pitch, c->P, i0, j0, w, h, static_cast<float *>(box));
    }
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_energy_box(qla_ctx *c, int i0, int j0, int w, int h) {
    if (c->prec == QLA_FP64)
        return c->P == 6 ? energy_box_p<double, 6>(c, i0, j0, w, h)
                         : energy_box_p<double, 3>(c, i0, j0, w, h);
    return c->P == 6 ? energy_box_p<float, 6>(c, i0, j0, w, h)
                     : energy_box_p<float, 3>(c, i0, j0, w, h);
}

cudaError_t launch_packet_window(qla_ctx *c, const qla_packet &p, int i0, int j0, int gnx,
                                 int gny) {
    if (c->prec == QLA_FP64)
        return c->P == 6 ? packet_window_p<double, 6>(c, p, i0, j0, gnx, gny)
                         : packet_window_p<double, 3>(c, p, i0, j0, gnx, gny);
    return c->P == 6 ? packet_window_p<float, 6>(c, p, i0, j0, gnx, gny)
                     : packet_window_p<float, 3>(c, p, i0, j0, gnx, gny);
}

}  // namespace qla
