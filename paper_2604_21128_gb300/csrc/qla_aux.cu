// Per-run kernels around the step: medium coefficients (Eqs. 2e4, 2e13),
// the initial packet (Sec. V-B), the energy reduction (Eq. A13), the inverse
// Dyson map to fields (Eq. 3b3) and FP64 <-> storage conversions.
#include "qla_internal.h"

namespace qla {
namespace {

constexpr int AUX_THREADS = 256;

inline int grid_for(size_t n, int threads = AUX_THREADS) {
    size_t b = (n + threads - 1) / threads;
    return int(b < 65535u * 32u ? (b > 0 ? b : 1) : 65535u * 32u);
}

// ---------------------------------------------------------------------------
// Medium: theta = delta/(4n) (Eq. 2e4); beta = delta^2 (dn/dx)/n^2 with the
// centred periodic difference (Eq. 2e13); V angle = beta/2 (rotation
// reading) or beta (printed shear).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void store_coef(double2 *cC, double4 *cV, size_t g, double th,
                                           double px, double py) {
    double s, c;
    sincos(th, &s, &c);
    cC[g] = make_double2(c, s);
    double sx, cx, sy, cy;
    sincos(px, &sx, &cx);
    sincos(py, &sy, &cy);
    cV[g] = make_double4(cx, sx, cy, sy);
}

__device__ __forceinline__ void split(double v, float &hi, float &lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - double(hi));
}

__device__ __forceinline__ void store_coef(float4 *cC, float4 *cV, size_t g, double th,
                                           double px, double py) {
    double s, c;
    sincos(th, &s, &c);
    float4 k;
    split(c, k.x, k.z);
    split(s, k.y, k.w);
    cC[g] = k;
    // gamma = 1 - cos = 2 sin^2(phi/2), computed without cancellation
    const double shx = sin(0.5 * px), shy = sin(0.5 * py);
    cV[g] = make_float4(__double2float_rn(2.0 * shx * shx), __double2float_rn(sin(px)),
                        __double2float_rn(2.0 * shy * shy), __double2float_rn(sin(py)));
}

template <typename T>
__global__ void k_medium(const double *__restrict__ n, int nx, int ny, int pitch, double delta,
                         double vscale, typename Coef<T>::C *cC, typename Coef<T>::V *cV) {
    const size_t N = size_t(nx) * ny;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        const size_t g = size_t(j) * pitch + i;
        const double nn = n[g];
        const double th = delta / (4.0 * nn);
        const double nxp = n[size_t(j) * pitch + wrap(i + 1, nx)];
        const double nxm = n[size_t(j) * pitch + wrap(i - 1, nx)];
        const double nyp = n[size_t(wrap(j + 1, ny)) * pitch + i];
        const double nym = n[size_t(wrap(j - 1, ny)) * pitch + i];
        const double bx = (nxp - nxm) / (2.0 * delta) / (nn * nn) * delta * delta;
        const double by = (nyp - nym) / (2.0 * delta) / (nn * nn) * delta * delta;
        store_coef(cC, cV, g, th, vscale * bx, vscale * by);
    }
}

// Copy a contiguous FP64 host-layout plane into the pitched n plane.
__global__ void k_pitch_copy(const double *__restrict__ src, double *__restrict__ dst, int nx,
                             int ny, int pitch) {
    const size_t N = size_t(nx) * ny;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        dst[size_t(j) * pitch + i] = src[t];
    }
}

// ---------------------------------------------------------------------------
// Packet (Sec. V-B): E_z Gaussian with plane-wave B; q2 = n E_z,
// q3 = sin(angle) q2, q4 = -cos(angle) q2, others zero.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double min_image(double x, double x0, double L) {
    double d = fmod(x - x0 + 0.5 * L, L);
    if (d < 0.0) d += L;
    return d - 0.5 * L;
}

template <typename T, int P>
__global__ void k_packet(const double *__restrict__ n, T *__restrict__ q, int nx, int ny,
                         int pitch, size_t plane_elems, double delta, qla_packet p, double cphi,
                         double sphi) {
    const size_t N = size_t(nx) * ny;
    const double Lx = nx * delta, Ly = ny * delta;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        const size_t g = size_t(j) * pitch + i;
        const double dx = min_image(i * delta, p.x0, Lx);
        const double dy = min_image(j * delta, p.y0, Ly);
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

// ---------------------------------------------------------------------------
// Conversions and fields.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_from_f64(const double *__restrict__ src, T *__restrict__ dst, int nx, int ny,
                           int pitch) {
    const size_t N = size_t(nx) * ny;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        dst[size_t(j) * pitch + i] = T(src[t]);
    }
}

// dst[t] = src / n (E components) or src (B components); src == null -> 0.
template <typename T>
__global__ void k_to_f64(const T *__restrict__ src, const double *__restrict__ n,
                         double *__restrict__ dst, int nx, int ny, int pitch) {
    const size_t N = size_t(nx) * ny;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        const size_t g = size_t(j) * pitch + i;
        double v = src ? double(src[g]) : 0.0;
        if (n) v /= n[g];
        dst[t] = v;
    }
}

// ---------------------------------------------------------------------------
// Energy: FP64 sum of q^2 over sites and live planes.  Fixed grid, fixed
// per-thread order, fixed tree: bitwise reproducible for a given lattice.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double warp_part[AUX_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_part[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = lane < AUX_THREADS / 32 ? warp_part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;  // valid in thread 0
}

template <typename T, int P>
__global__ void __launch_bounds__(AUX_THREADS)
k_energy_partial(const T *__restrict__ q, int nx, int ny, int pitch, size_t plane_elems,
                 double *__restrict__ partials) {
    const size_t N = size_t(nx) * ny;
    double acc = 0.0;
    for (size_t t = blockIdx.x * size_t(AUX_THREADS) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * AUX_THREADS) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        const size_t g = size_t(j) * pitch + i;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const double v = double(q[p * plane_elems + g]);
            acc = fma(v, v, acc);
        }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(AUX_THREADS)
k_energy_final(const double *__restrict__ partials, int count, double *__restrict__ out) {
    double acc = 0.0;
    for (int t = threadIdx.x; t < count; t += AUX_THREADS) acc += partials[t];
    acc = block_sum(acc);
    if (threadIdx.x == 0) *out = acc;
}

// Gather q at listed sites: ij holds i[0..count) then j[0..count).
template <typename T, int P>
__global__ void k_probe(const T *__restrict__ q, const int *__restrict__ ij, int count,
                        int pitch, size_t plane_elems, double *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const size_t g = size_t(ij[count + k]) * pitch + ij[k];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const int p = plane_of<P>(c);
        out[6 * k + c] = p >= 0 ? double(q[p * plane_elems + g]) : 0.0;
    }
}

}  // namespace

cudaError_t launch_probe(qla_ctx *c, int count, const int *ij_dev, double *out_dev) {
    const int nb = (count + AUX_THREADS - 1) / AUX_THREADS;
    const void *q = c->state[c->cur];
    if (c->prec == QLA_FP64) {
        if (c->P == 6)
            k_probe<double, 6><<<nb, AUX_THREADS, 0, c->stream>>>(
                static_cast<const double *>(q), ij_dev, count, c->pitch, c->plane_elems, out_dev);
        else
            k_probe<double, 3><<<nb, AUX_THREADS, 0, c->stream>>>(
                static_cast<const double *>(q), ij_dev, count, c->pitch, c->plane_elems, out_dev);
    } else {
        if (c->P == 6)
            k_probe<float, 6><<<nb, AUX_THREADS, 0, c->stream>>>(
                static_cast<const float *>(q), ij_dev, count, c->pitch, c->plane_elems, out_dev);
        else
            k_probe<float, 3><<<nb, AUX_THREADS, 0, c->stream>>>(
                static_cast<const float *>(q), ij_dev, count, c->pitch, c->plane_elems, out_dev);
    }
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_medium(qla_ctx *c) {
    const size_t N = size_t(c->nx) * c->ny;
    // host n was staged contiguously; place it in the pitched plane first
    k_pitch_copy<<<grid_for(N), AUX_THREADS, 0, c->stream>>>(c->staging, c->n, c->nx, c->ny,
                                                              c->pitch);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double vscale = c->vmode == V_ROTATION ? 0.5 : 1.0;
    if (c->prec == QLA_FP64)
        k_medium<double><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(
            c->n, c->nx, c->ny, c->pitch, c->delta, vscale,
            static_cast<double2 *>(c->coefC), static_cast<double4 *>(c->coefV));
    else
        k_medium<float><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(
            c->n, c->nx, c->ny, c->pitch, c->delta, vscale, static_cast<float4 *>(c->coefC),
            static_cast<float4 *>(c->coefV));
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_packet(qla_ctx *c, const qla_packet &p) {
    const size_t N = size_t(c->nx) * c->ny;
    const double cphi = cos(p.angle), sphi = sin(p.angle);
    void *q = c->state[c->cur];
    if (c->prec == QLA_FP64) {
        if (c->P == 6)
            k_packet<double, 6><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(
                c->n, static_cast<double *>(q), c->nx, c->ny, c->pitch, c->plane_elems,
                c->delta, p, cphi, sphi);
        else
            k_packet<double, 3><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(
                c->n, static_cast<double *>(q), c->nx, c->ny, c->pitch, c->plane_elems,
                c->delta, p, cphi, sphi);
    } else {
        if (c->P == 6)
            k_packet<float, 6><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(
                c->n, static_cast<float *>(q), c->nx, c->ny, c->pitch, c->plane_elems,
                c->delta, p, cphi, sphi);
        else
            k_packet<float, 3><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(
                c->n, static_cast<float *>(q), c->nx, c->ny, c->pitch, c->plane_elems,
                c->delta, p, cphi, sphi);
    }
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_from_f64(qla_ctx *c, int plane, const double *src) {
    const size_t N = size_t(c->nx) * c->ny;
    if (c->prec == QLA_FP64)
        k_from_f64<double><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(
            src, static_cast<double *>(c->state[c->cur]) + plane * c->plane_elems, c->nx, c->ny,
            c->pitch);
    else
        k_from_f64<float><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(
            src, static_cast<float *>(c->state[c->cur]) + plane * c->plane_elems, c->nx, c->ny,
            c->pitch);
    c->launches++;
    return cudaGetLastError();
}

static cudaError_t to_f64(qla_ctx *c, int plane, const double *n, double *dst) {
    const size_t N = size_t(c->nx) * c->ny;
    if (c->prec == QLA_FP64) {
        const double *src =
            plane >= 0 ? static_cast<const double *>(c->state[c->cur]) + plane * c->plane_elems
                       : nullptr;
        k_to_f64<double><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(src, n, dst, c->nx, c->ny,
                                                                      c->pitch);
    } else {
        const float *src =
            plane >= 0 ? static_cast<const float *>(c->state[c->cur]) + plane * c->plane_elems
                       : nullptr;
        k_to_f64<float><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(src, n, dst, c->nx, c->ny,
                                                                     c->pitch);
    }
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_to_f64(qla_ctx *c, int plane, double *dst) {
    return to_f64(c, plane, nullptr, dst);
}

cudaError_t launch_fields(qla_ctx *c, int comp, double *dst) {
    const int plane = c->P == 6 ? comp : plane_of<3>(comp);
    return to_f64(c, plane, comp < 3 ? c->n : nullptr, dst);
}

cudaError_t launch_energy(qla_ctx *c) {
    const void *q = c->state[c->cur];
    const int nb = c->energy_blocks;
    if (c->prec == QLA_FP64) {
        if (c->P == 6)
            k_energy_partial<double, 6><<<nb, AUX_THREADS, 0, c->stream>>>(
                static_cast<const double *>(q), c->nx, c->ny, c->pitch, c->plane_elems,
                c->partials);
        else
            k_energy_partial<double, 3><<<nb, AUX_THREADS, 0, c->stream>>>(
                static_cast<const double *>(q), c->nx, c->ny, c->pitch, c->plane_elems,
                c->partials);
    } else {
        if (c->P == 6)
            k_energy_partial<float, 6><<<nb, AUX_THREADS, 0, c->stream>>>(
                static_cast<const float *>(q), c->nx, c->ny, c->pitch, c->plane_elems,
                c->partials);
        else
            k_energy_partial<float, 3><<<nb, AUX_THREADS, 0, c->stream>>>(
                static_cast<const float *>(q), c->nx, c->ny, c->pitch, c->plane_elems,
                c->partials);
    }
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_energy_final<<<1, AUX_THREADS, 0, c->stream>>>(c->partials, nb, c->result);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace qla
