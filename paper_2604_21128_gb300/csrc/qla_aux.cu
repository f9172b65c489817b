// Per-run kernels around the step: medium coefficients (Eqs. 2e4, 2e13),
// the initial packet (Sec. V-B), the energy reduction (Eq. A13), the inverse
// Dyson map to fields (Eq. 3b3) and FP64 <-> storage conversions.
#include <cooperative_groups.h>

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
__device__ __forceinline__ void make_rec(MedRec<double> &r, double th, double px, double py) {
    // collision: (tan(theta/2), sin theta) for the three-shear rotation
    r.c = make_double2(tan(0.5 * th), sin(th));
    double sx, cx, sy, cy;
    sincos(px, &sx, &cx);
    sincos(py, &sy, &cy);
    r.v = make_double4_16a(cx, sx, cy, sy);
}

__device__ __forceinline__ void split(double v, float &hi, float &lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - double(hi));
}

__device__ __forceinline__ void make_rec(MedRec<float> &r, double th, double px, double py) {
    double s, c;
    sincos(th, &s, &c);
    split(c, r.c.x, r.c.z);
    split(s, r.c.y, r.c.w);
    // gamma = 1 - cos = 2 sin^2(phi/2), computed without cancellation
    const double shx = sin(0.5 * px), shy = sin(0.5 * py);
    r.v = make_float4(__double2float_rn(2.0 * shx * shx), __double2float_rn(sin(px)),
                      __double2float_rn(2.0 * shy * shy), __double2float_rn(sin(py)));
}

// An FP64 value as three FP32 words whose exact sum it is.
__device__ __forceinline__ void split3(double v, float &a, float &b, float &c) {
    a = __double2float_rn(v);
    const double r = v - double(a);
    b = __double2float_rn(r);
    c = __double2float_rn(r - double(b));
}

__device__ __forceinline__ void split3(double cv, double sv, DSCoef &k) {
    split3(cv, k.c0, k.c1, k.c2);
    split3(sv, k.s0, k.s1, k.s2);
    k.pad0 = k.pad1 = 0.0f;
}

// Double-single records: the FP64 record's cosines and sines, three words each.
__device__ __forceinline__ void make_rec(MedRec<dsf> &r, double th, double px, double py) {
    double s, c;
    sincos(th, &s, &c);
    split3(c, s, r.c);
    double sx, cx, sy, cy;
    sincos(px, &sx, &cx);
    sincos(py, &sy, &cy);
    split3(cx, sx, r.v.x);
    split3(cy, sy, r.v.y);
}

// One pass over the sites: classify, hand out a record index, write each
// record once.  A site whose four neighbours carry exactly its n has beta = 0
// and a record that depends on n alone; those share one record per distinct
// n through an open-addressing table of UNIFORM_SLOTS keys (n's bits; n > 0
// so a key is never 0, the empty mark).  The site that claims a key writes
// its record.  All other sites get consecutive fresh indices after the
// shared slots (one atomic per group of lanes) and write their own record.
// Index values depend on scheduling; record contents do not, so results are
// reproducible bit for bit.
template <typename T>
__global__ void k_medium(const double *__restrict__ n, int nx, int ny, int pitch, double delta,
                         double vscale, unsigned long long *__restrict__ keys,
                         unsigned *__restrict__ counter, uint32_t *__restrict__ midx,
                         MedRec<T> *__restrict__ table, MedRec<dsf> *__restrict__ ds_table) {
    namespace cg = cooperative_groups;
    const size_t N = size_t(nx) * ny;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        const size_t g = size_t(j) * pitch + i;
        const double nn = n[g];
        const double nxp = n[size_t(j) * pitch + wrap(i + 1, nx)];
        const double nxm = n[size_t(j) * pitch + wrap(i - 1, nx)];
        const double nyp = n[size_t(wrap(j + 1, ny)) * pitch + i];
        const double nym = n[size_t(wrap(j - 1, ny)) * pitch + i];
        bool shared = nxp == nn && nxm == nn && nyp == nn && nym == nn;
        bool owner = false;
        uint32_t id = 0;
        if (shared) {
            const unsigned long long key = static_cast<unsigned long long>(__double_as_longlong(nn));
            unsigned h = unsigned(mix64(key)) & (UNIFORM_SLOTS - 1);
            bool placed = false;
            for (int probe = 0; probe < UNIFORM_SLOTS; ++probe) {
                // a plateau's key is placed by its first site; the others find
                // it with a plain read instead of all contending for one atomic
                // (16384^2 bubble: 168 ms with every site's atomicCAS)
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
            const double th = delta / (4.0 * nn);
            const double bx = (nxp - nxm) / (2.0 * delta) / (nn * nn) * delta * delta;
            const double by = (nyp - nym) / (2.0 * delta) / (nn * nn) * delta * delta;
            MedRec<T> r;
            make_rec(r, th, vscale * bx, vscale * by);
            table[id] = r;
            if (ds_table) {   // QLA_DOUBLE_SINGLE: the same record in word triples
                MedRec<dsf> rd;
                make_rec(rd, th, vscale * bx, vscale * by);
                ds_table[id] = rd;
            }
        }
        midx[g] = id;
    }
}

// Copy a contiguous FP64 host-layout plane into the pitched n plane.
// Records of a diagonal index tensor, one per stored site: each pair's
// collision angle from its own component (Eqs. 2e4, 2e8) and the potential
// angles beta_0..beta_3 of Eq. 2e13 (centred periodic differences), times
// vscale (1/2 for the rotation reading).  The same coefficient construction
// as the scalar records (make_rec).
template <typename T>
__global__ void k_medium_tensor(const double *__restrict__ nX, const double *__restrict__ nY,
                                const double *__restrict__ nZ, int nx, int ny, int pitch,
                                double delta, double vscale, MedRecT<T> *__restrict__ table) {
    const size_t N = size_t(nx) * ny;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        const size_t g = size_t(j) * pitch + i;
        const size_t gxp = size_t(j) * pitch + wrap(i + 1, nx), gxm = size_t(j) * pitch + wrap(i - 1, nx);
        const size_t gyp = size_t(wrap(j + 1, ny)) * pitch + i, gym = size_t(wrap(j - 1, ny)) * pitch + i;
        const double ax = nX[g], ay = nY[g], az = nZ[g];
        // the expression of k_medium, so equal components give equal records
        const double b0 = (nY[gxp] - nY[gxm]) / (2.0 * delta) / (ay * ay) * delta * delta;
        const double b2 = (nZ[gxp] - nZ[gxm]) / (2.0 * delta) / (az * az) * delta * delta;
        const double b1 = (nX[gyp] - nX[gym]) / (2.0 * delta) / (ax * ax) * delta * delta;
        const double b3 = (nZ[gyp] - nZ[gym]) / (2.0 * delta) / (az * az) * delta * delta;
        MedRec<T> ry, rz, rx;
        make_rec(ry, delta / (4.0 * ay), vscale * b0, vscale * b1);
        make_rec(rz, delta / (4.0 * az), vscale * b2, vscale * b3);
        make_rec(rx, delta / (4.0 * ax), 0.0, 0.0);
        MedRecT<T> r;
        r.c15 = ry.c;
        r.c2 = rz.c;
        r.c05 = rx.c;
        r.vz = rz.v;
        r.vt = ry.v;
        table[g] = r;
    }
}

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

// dst[t] = q_comp / n (with n) or q_comp, where q is the state at the site
// (pending potential operator applied; absent planes read as zero).
template <typename T, int P, int VM>
__global__ void k_to_f64(const T *__restrict__ q, size_t plane_elems, int comp,
                         const double *__restrict__ n, double *__restrict__ dst, int nx, int ny,
                         int pitch, bool vin, const uint32_t *__restrict__ midx,
                         const MedRec<T> *__restrict__ table) {
    const size_t N = size_t(nx) * ny;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        const size_t g = size_t(j) * pitch + i;
        T s[6];
        load_site<T, P, VM>(q, plane_elems, g, vin, midx, table, s);
        double v = double(s[comp]);
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
    __syncthreads();  // warp_part is reused by the next call
    return v;  // valid in thread 0
}

template <typename T, int P, int VM>
__global__ void __launch_bounds__(AUX_THREADS)
k_energy_partial(const T *__restrict__ q, int nx, int ny, int pitch, size_t plane_elems,
                 double *__restrict__ partials, bool vin, const uint32_t *__restrict__ midx,
                 const MedRec<T> *__restrict__ table) {
    const size_t N = size_t(nx) * ny;
    double acc = 0.0;
    for (size_t t = blockIdx.x * size_t(AUX_THREADS) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * AUX_THREADS) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        const size_t g = size_t(j) * pitch + i;
        T s[6];
        load_site<T, P, VM>(q, plane_elems, g, vin, midx, table, s);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (plane_of<P>(c) < 0) continue;
            const double v = double(s[c]);
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

__device__ double block_max(double v) {
    __shared__ double warp_part[AUX_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) warp_part[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = lane < AUX_THREADS / 32 ? warp_part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;  // valid in thread 0
}

// Gauss laws (Eqs. 3.1, 3.2) with centred periodic differences: fields vary
// in x and y only, B = (q3, q4), D = (n_x q0, n_y q1) (Dyson variables,
// c = 1; n_x = n_y = n for a scalar medium).  Each site reads its four neighbours' amplitudes (the pending
// potential step applied) and medium.
template <typename T, int P, int VM>
__global__ void __launch_bounds__(AUX_THREADS)
k_div_partial(const T *__restrict__ q, const double *__restrict__ nX,
              const double *__restrict__ nY, int nx, int ny, int pitch,
              size_t plane_elems, double inv2d, double *__restrict__ partials, bool vin,
              const uint32_t *__restrict__ midx, const MedRec<T> *__restrict__ table) {
    const size_t N = size_t(nx) * ny;
    double sb = 0.0, gb = 0.0, sd = 0.0, gd = 0.0, mb = 0.0, md = 0.0;
    for (size_t t = blockIdx.x * size_t(AUX_THREADS) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * AUX_THREADS) {
        const int j = int(t / nx), i = int(t - size_t(j) * nx);
        const size_t gxp = size_t(j) * pitch + wrap(i + 1, nx);
        const size_t gxm = size_t(j) * pitch + wrap(i - 1, nx);
        const size_t gyp = size_t(wrap(j + 1, ny)) * pitch + i;
        const size_t gym = size_t(wrap(j - 1, ny)) * pitch + i;
        T a[6], b[6], c[6], d[6];
        load_site<T, P, VM>(q, plane_elems, gxp, vin, midx, table, a);
        load_site<T, P, VM>(q, plane_elems, gxm, vin, midx, table, b);
        load_site<T, P, VM>(q, plane_elems, gyp, vin, midx, table, c);
        load_site<T, P, VM>(q, plane_elems, gym, vin, midx, table, d);
        const double dbx = inv2d * (double(a[3]) - double(b[3]));
        const double dby = inv2d * (double(c[4]) - double(d[4]));
        const double ddx = inv2d * (nX[gxp] * double(a[0]) - nX[gxm] * double(b[0]));
        const double ddy = inv2d * (nY[gyp] * double(c[1]) - nY[gym] * double(d[1]));
        const double db = dbx + dby, dd = ddx + ddy;
        sb = fma(db, db, sb);
        gb = fma(dbx, dbx, fma(dby, dby, gb));
        sd = fma(dd, dd, sd);
        gd = fma(ddx, ddx, fma(ddy, ddy, gd));
        mb = fmax(mb, fabs(db));
        md = fmax(md, fabs(dd));
    }
    const double r[DIV_TERMS] = {block_sum(sb), block_sum(gb), block_sum(sd), block_sum(gd),
                                 block_max(mb), block_max(md)};
    if (threadIdx.x == 0)
        for (int k = 0; k < DIV_TERMS; ++k) partials[size_t(blockIdx.x) * DIV_TERMS + k] = r[k];
}

__global__ void __launch_bounds__(AUX_THREADS)
k_div_final(const double *__restrict__ partials, int count, double *__restrict__ out) {
    double v[DIV_TERMS] = {0, 0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < count; t += AUX_THREADS)
        for (int k = 0; k < DIV_TERMS; ++k) {
            const double p = partials[size_t(t) * DIV_TERMS + k];
            v[k] = k < 4 ? v[k] + p : fmax(v[k], p);
        }
    double r[DIV_TERMS];
    for (int k = 0; k < DIV_TERMS; ++k) r[k] = k < 4 ? block_sum(v[k]) : block_max(v[k]);
    if (threadIdx.x == 0)
        for (int k = 0; k < DIV_TERMS; ++k) out[k] = r[k];
}

// Gather q at listed sites: ij holds i[0..count) then j[0..count).
template <typename T, int P, int VM>
__global__ void k_probe(const T *__restrict__ q, const int *__restrict__ ij, int count,
                        int pitch, size_t plane_elems, double *__restrict__ out, bool vin,
                        const uint32_t *__restrict__ midx, const MedRec<T> *__restrict__ table) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const size_t g = size_t(ij[count + k]) * pitch + ij[k];
    T s[6];
    load_site<T, P, VM>(q, plane_elems, g, vin, midx, table, s);
#pragma unroll
    for (int c = 0; c < 6; ++c) out[6 * k + c] = double(s[c]);
}

}  // namespace

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
            c->n, c->nx, c->ny, c->pitch, c->delta, vscale, c->keys, c->counter, c->midx,
            static_cast<MedRec<double> *>(c->table), static_cast<MedRec<dsf> *>(c->dstable));
    else
        k_medium<float><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(
            c->n, c->nx, c->ny, c->pitch, c->delta, vscale, c->keys, c->counter, c->midx,
            static_cast<MedRec<float> *>(c->table), nullptr);
    c->launches++;
    return cudaGetLastError();
}

// QLA_DOUBLE_SINGLE: the state buffer between FP64 and word pairs, in place
// (each 8-byte element is read and rewritten by one thread).
__global__ void k_to_ds(double *__restrict__ q, size_t n) {
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < n;
         t += size_t(gridDim.x) * blockDim.x) {
        const double v = q[t];
        const float hi = __double2float_rn(v);
        const float lo = __double2float_rn(v - double(hi));
        reinterpret_cast<float2 *>(q)[t] = make_float2(hi, lo);
    }
}

__global__ void k_from_ds(double *__restrict__ q, size_t n) {
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < n;
         t += size_t(gridDim.x) * blockDim.x) {
        const float2 w = reinterpret_cast<const float2 *>(q)[t];
        q[t] = double(w.x) + double(w.y);
    }
}

cudaError_t raw_to_ds(void *q, size_t n, cudaStream_t st) {
    k_to_ds<<<grid_for(n), AUX_THREADS, 0, st>>>(static_cast<double *>(q), n);
    return cudaGetLastError();
}

cudaError_t raw_from_ds(void *q, size_t n, cudaStream_t st) {
    k_from_ds<<<grid_for(n), AUX_THREADS, 0, st>>>(static_cast<double *>(q), n);
    return cudaGetLastError();
}

cudaError_t launch_state_to_ds(qla_ctx *c, void *state) {
    return raw_to_ds(state, size_t(c->P) * c->plane_elems, c->stream);
}

cudaError_t launch_state_from_ds(qla_ctx *c, void *state) {
    return raw_from_ds(state, size_t(c->P) * c->plane_elems, c->stream);
}

// Raw-pointer forms of the conversions and the energy for a six-plane state
// with no pending potential step (the three-dimensional path, whose
// lattice is nx x rows with rows = ny * nz).
cudaError_t raw_pitch_copy(const double *src, double *dst, int nx, int rows, int pitch,
                           cudaStream_t st) {
    k_pitch_copy<<<grid_for(size_t(nx) * rows), AUX_THREADS, 0, st>>>(src, dst, nx, rows, pitch);
    return cudaGetLastError();
}

cudaError_t raw_from_f64(int prec, const double *src, void *plane, int nx, int rows, int pitch,
                         cudaStream_t st) {
    const size_t N = size_t(nx) * rows;
    if (prec == QLA_FP64)
        k_from_f64<double><<<grid_for(N), AUX_THREADS, 0, st>>>(src, static_cast<double *>(plane),
                                                                 nx, rows, pitch);
    else
        k_from_f64<float><<<grid_for(N), AUX_THREADS, 0, st>>>(src, static_cast<float *>(plane),
                                                                nx, rows, pitch);
    return cudaGetLastError();
}

cudaError_t raw_to_f64(int prec, const void *state, size_t plane_elems, int comp, double *dst,
                       int nx, int rows, int pitch, cudaStream_t st) {
    const size_t N = size_t(nx) * rows;
    if (prec == QLA_FP64)
        k_to_f64<double, 6, V_NONE><<<grid_for(N), AUX_THREADS, 0, st>>>(
            static_cast<const double *>(state), plane_elems, comp, nullptr, dst, nx, rows, pitch,
            false, nullptr, nullptr);
    else
        k_to_f64<float, 6, V_NONE><<<grid_for(N), AUX_THREADS, 0, st>>>(
            static_cast<const float *>(state), plane_elems, comp, nullptr, dst, nx, rows, pitch,
            false, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t raw_energy(int prec, const void *state, size_t plane_elems, int nx, int rows,
                       int pitch, double *partials, int nblocks, double *result, cudaStream_t st) {
    if (prec == QLA_FP64)
        k_energy_partial<double, 6, V_NONE><<<nblocks, AUX_THREADS, 0, st>>>(
            static_cast<const double *>(state), nx, rows, pitch, plane_elems, partials, false,
            nullptr, nullptr);
    else
        k_energy_partial<float, 6, V_NONE><<<nblocks, AUX_THREADS, 0, st>>>(
            static_cast<const float *>(state), nx, rows, pitch, plane_elems, partials, false,
            nullptr, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_energy_final<<<1, AUX_THREADS, 0, st>>>(partials, nblocks, result);
    return cudaGetLastError();
}

cudaError_t launch_pitch_copy(qla_ctx *c, double *dst) {
    const size_t N = size_t(c->nx) * c->ny;
    k_pitch_copy<<<grid_for(N), AUX_THREADS, 0, c->stream>>>(c->staging, dst, c->nx, c->ny,
                                                              c->pitch);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_medium_tensor(qla_ctx *c) {
    const size_t N = size_t(c->nx) * c->ny;
    const double vscale = c->vmode == V_ROTATION ? 0.5 : 1.0;
    if (c->prec == QLA_FP64)
        k_medium_tensor<double><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(
            c->n_x, c->n_y, c->n, c->nx, c->ny, c->pitch, c->delta, vscale,
            static_cast<MedRecT<double> *>(c->ttable));
    else
        k_medium_tensor<float><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(
            c->n_x, c->n_y, c->n, c->nx, c->ny, c->pitch, c->delta, vscale,
            static_cast<MedRecT<float> *>(c->ttable));
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

// Read-out launchers: one instantiation per (precision, planes, V reading).
template <typename T, int P, int VM>
static cudaError_t readout_t(qla_ctx *c, int what, int comp, const double *n, double *dst,
                             int count, const int *ij) {
    const size_t N = size_t(c->nx) * c->ny;
    const T *q = static_cast<const T *>(c->state[c->cur]);
    const MedRec<T> *table = static_cast<const MedRec<T> *>(c->table);
    const bool vin = c->pending_v;
    if (what == 0) {
        k_to_f64<T, P, VM><<<grid_for(N), AUX_THREADS, 0, c->stream>>>(
            q, c->plane_elems, comp, n, dst, c->nx, c->ny, c->pitch, vin, c->midx, table);
    } else if (what == 1) {
        k_energy_partial<T, P, VM><<<c->energy_blocks, AUX_THREADS, 0, c->stream>>>(
            q, c->nx, c->ny, c->pitch, c->plane_elems, c->partials, vin, c->midx, table);
    } else {
        k_probe<T, P, VM><<<(count + AUX_THREADS - 1) / AUX_THREADS, AUX_THREADS, 0, c->stream>>>(
            q, ij, count, c->pitch, c->plane_elems, dst, vin, c->midx, table);
    }
    c->launches++;
    return cudaGetLastError();
}

template <typename T, int P>
static cudaError_t readout_p(qla_ctx *c, int what, int comp, const double *n, double *dst,
                             int count, const int *ij) {
    switch (c->vmode) {
    case V_ROTATION: return readout_t<T, P, V_ROTATION>(c, what, comp, n, dst, count, ij);
    case V_LITERAL:  return readout_t<T, P, V_LITERAL>(c, what, comp, n, dst, count, ij);
    default:         return readout_t<T, P, V_NONE>(c, what, comp, n, dst, count, ij);
    }
}

static cudaError_t readout(qla_ctx *c, int what, int comp, const double *n, double *dst,
                           int count = 0, const int *ij = nullptr) {
    if (c->prec == QLA_FP64)
        return c->P == 6 ? readout_p<double, 6>(c, what, comp, n, dst, count, ij)
                         : readout_p<double, 3>(c, what, comp, n, dst, count, ij);
    return c->P == 6 ? readout_p<float, 6>(c, what, comp, n, dst, count, ij)
                     : readout_p<float, 3>(c, what, comp, n, dst, count, ij);
}

cudaError_t launch_to_f64(qla_ctx *c, int comp, double *dst) {
    return readout(c, 0, comp, nullptr, dst);
}

cudaError_t launch_fields(qla_ctx *c, int comp, double *dst) {
    const double *n = comp == 0 && c->tensor ? c->n_x
                    : comp == 1 && c->tensor ? c->n_y
                    : comp < 3              ? c->n
                                            : nullptr;
    return readout(c, 0, comp, n, dst);
}

cudaError_t launch_probe(qla_ctx *c, int count, const int *ij_dev, double *out_dev) {
    return readout(c, 2, 0, nullptr, out_dev, count, ij_dev);
}

template <typename T, int P, int VM>
static cudaError_t divergence_t(qla_ctx *c) {
    k_div_partial<T, P, VM><<<c->energy_blocks, AUX_THREADS, 0, c->stream>>>(
        static_cast<const T *>(c->state[c->cur]), c->tensor ? c->n_x : c->n,
        c->tensor ? c->n_y : c->n, c->nx, c->ny, c->pitch, c->plane_elems,
        0.5 / c->delta, c->partials, c->pending_v, c->midx,
        static_cast<const MedRec<T> *>(c->table));
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_div_final<<<1, AUX_THREADS, 0, c->stream>>>(c->partials, c->energy_blocks, c->result);
    c->launches++;
    return cudaGetLastError();
}

template <typename T, int P>
static cudaError_t divergence_p(qla_ctx *c) {
    switch (c->vmode) {
    case V_ROTATION: return divergence_t<T, P, V_ROTATION>(c);
    case V_LITERAL:  return divergence_t<T, P, V_LITERAL>(c);
    default:         return divergence_t<T, P, V_NONE>(c);
    }
}

cudaError_t launch_divergence(qla_ctx *c) {
    if (c->prec == QLA_FP64) return c->P == 6 ? divergence_p<double, 6>(c) : divergence_p<double, 3>(c);
    return c->P == 6 ? divergence_p<float, 6>(c) : divergence_p<float, 3>(c);
}

cudaError_t launch_energy(qla_ctx *c) {
    cudaError_t e = readout(c, 1, 0, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    k_energy_final<<<1, AUX_THREADS, 0, c->stream>>>(c->partials, c->energy_blocks, c->result);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace qla
