// Energy of caller-owned state planes with no device allocation: the
// reduction's partial sums live in a fixed file-scope device array instead of
// a workspace.  For callers that cannot allocate device memory (see
// qla_energy_noalloc in include/qla.h).
#include <atomic>
#include <mutex>

#include "qla_internal.h"

namespace qla {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_DEVICES = 64;

// Scratch shared by every call in the process, on every device that loads
// the library (it stays allocated until the process exits).  A call writes
// partials[0 .. blocks) before the final pass reads them, so nothing needs
// clearing between calls; two calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_noalloc_partials[QLA_NOALLOC_MAX_PARTIALS];

// Device address of the scratch, looked up once per device.  Host code may
// not pass &g_noalloc_partials to a kernel: on the host that name is a
// host-side stand-in, not a device address.
std::mutex g_addr_mutex;
double *g_addr[NA_MAX_DEVICES] = {};

cudaError_t scratch_for(int dev, double **out) {
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

__device__ __forceinline__ double na_block_sum(double v) {
    __shared__ double part[NA_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = lane < NA_THREADS / 32 ? part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// Block b sums q^2 over sites [b*S, (b+1)*S) of every plane, S =
// QLA_NOALLOC_SITES_PER_PARTIAL, in a fixed order: row by row (the block's
// range splits into whole rows plus a partial first and last row), the
// threads striding along each row.
template <typename T>
__global__ void __launch_bounds__(NA_THREADS)
k_na_partial(const T *__restrict__ q, int planes, int nx, long long sites, long long pitch,
             long long stride, double *__restrict__ partials) {
    const long long s0 = (long long)blockIdx.x * QLA_NOALLOC_SITES_PER_PARTIAL;
    long long s1 = s0 + QLA_NOALLOC_SITES_PER_PARTIAL;
    if (s1 > sites) s1 = sites;
    double acc = 0.0;
    const long long j0 = s0 / nx, j1 = (s1 - 1) / nx;
    for (long long j = j0; j <= j1; ++j) {
        const long long rs = j * nx;
        const long long a = (s0 > rs ? s0 : rs) - rs;
        const long long b = (s1 < rs + nx ? s1 : rs + nx) - rs;
        const T *row = q + j * pitch;
        for (long long i = a + threadIdx.x; i < b; i += NA_THREADS) {
            for (int p = 0; p < planes; ++p) {
                const double v = double(row[p * stride + i]);
                acc = fma(v, v, acc);
            }
        }
    }
    acc = na_block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(NA_THREADS)
k_na_final(const double *__restrict__ partials, int count, double *__restrict__ out) {
    double acc = 0.0;
    for (int t = threadIdx.x; t < count; t += NA_THREADS) acc += partials[t];
    acc = na_block_sum(acc);
    if (threadIdx.x == 0) *out = acc;
}

}  // namespace
}  // namespace qla

extern "C" qla_status qla_energy_noalloc(const void *planes, int precision, int n_planes, int nx,
                                         int ny, long long row_pitch, long long plane_stride,
                                         void *cuda_stream, double *out_dev) {
    using namespace qla;
    if (!planes || !out_dev) return QLA_EINVAL;
    if (precision != QLA_FP64 && precision != QLA_FP32) return QLA_EINVAL;
    if (n_planes < 1 || n_planes > 6 || nx < 1 || ny < 1) return QLA_EINVAL;
    if (row_pitch < nx || plane_stride < row_pitch * (long long)ny) return QLA_EINVAL;
    const long long sites = (long long)nx * ny;
    const long long blocks =
        (sites + QLA_NOALLOC_SITES_PER_PARTIAL - 1) / QLA_NOALLOC_SITES_PER_PARTIAL;
    if (blocks > QLA_NOALLOC_MAX_PARTIALS) return QLA_EINVAL;  // beyond the fixed scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QLA_ECUDA;
    double *partials = nullptr;
    if (scratch_for(dev, &partials) != cudaSuccess) return QLA_ECUDA;
    // An error another caller left pending is not ours to report or clear:
    // refuse without launching and leave it in place.  Any error after the
    // launches below is then this call's own.
    if (cudaPeekAtLastError() != cudaSuccess) return QLA_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (precision == QLA_FP64)
        k_na_partial<double><<<int(blocks), NA_THREADS, 0, st>>>(
            static_cast<const double *>(planes), n_planes, nx, sites, row_pitch, plane_stride,
            partials);
    else
        k_na_partial<float><<<int(blocks), NA_THREADS, 0, st>>>(
            static_cast<const float *>(planes), n_planes, nx, sites, row_pitch, plane_stride,
            partials);
    if (cudaGetLastError() != cudaSuccess) return QLA_ECUDA;
    k_na_final<<<1, NA_THREADS, 0, st>>>(partials, int(blocks), out_dev);
    if (cudaGetLastError() != cudaSuccess) return QLA_ECUDA;
    return QLA_OK;
}
