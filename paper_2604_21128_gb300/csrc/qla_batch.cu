// Batched lattices: many independent QLA lattices advanced together by one
// persistent, cooperative kernel per chunk of steps (declared in qla.h).
//
// Work is a flat list of items -- (instance, column window, row segment) --
// of similar cost whatever the lattice sizes.  Each warp of a grid sized to
// be fully co-resident takes items from a shared counter as it frees up and
// runs the marching step on them (qla_march.cuh); after each step the grid
// meets at a barrier so that the next step reads finished rows.  The
// barrier's wait is bounded: a block
// that waits longer than the budget raises an error word and every block
// leaves, and the host reports QLA_ETIMEOUT.  qla_batch_run captures a whole
// run (step chunks and batched energy reductions) as one CUDA graph.
#include <algorithm>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "qla_limits.h"
#include "qla_march2.cuh"
#include "qla_plateau.cuh"

namespace qla {
namespace {

using namespace march;

struct BatchInst {
    void *buf[2];          // the two state buffers (plane 0, row 0)
    const uint32_t *midx;
    const void *table;
    int nx, ny, pitch, seg, n_wx;
    uint32_t plane, total;
    int cur;               // buffer holding the state when the run starts
    int vin;               // a potential operator is pending at the start
};

struct BatchItem {
    int inst, item;
};

// A unit of the plateau-split FP32 E_z kernel (qla_plateau.cuh) and its
// instance.
struct BatchUnit {
    int4 u;
    int inst, pad0, pad1, pad2;
};

struct Barrier {
    unsigned count;        // blocks arrived at the current barrier
    unsigned gen;          // barriers completed
    unsigned next[2];      // next work item of the steps of even / odd parity
    int err;               // set when a wait ran out
    int pad;
};

constexpr int ENERGY_BLOCKS = 64;   // partial sums per instance
constexpr int ENERGY_ROWS = 64;     // energy rows kept on the device per graph

// Grid-wide barrier for a co-resident grid.  One thread per block arrives;
// the last arrival advances the generation.  The others wait for that with a
// bounded spin; on expiry they raise err, and every block sees err and
// leaves.  Returns false if the grid must stop.
__device__ __forceinline__ bool grid_barrier(Barrier *b, long long budget, bool skip) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &b->gen;
        volatile int *err = &b->err;
        const unsigned g = *gen;
        __threadfence();
        if (!skip) {
            const unsigned prev = atomicAdd(&b->count, 1u);
            if (prev == gridDim.x - 1) {
                b->count = 0;
                __threadfence();
                atomicAdd(&b->gen, 1u);
            }
        }
        const long long t0 = clock64();
        while (*gen == g && *err == 0) {
            if (clock64() - t0 > budget) {
                atomicExch(&b->err, 1);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
    return *static_cast<volatile int *>(&b->err) == 0;
}

// The marching machinery of a lane layout: LX adjacent columns per lane, or
// LX = 1 for the packed pairs of FP32 E_z lattices (qla_march2.cuh).
template <typename T, int P, int LX, int VM, bool VIN> struct MarchOf {
    using type = March<T, P, LX, VM, VIN>;
};
template <int VM, bool VIN> struct MarchOf<float, 3, 1, VM, VIN> {
    using type = March2<VM, VIN, PairF2>;
};

template <typename T, int P, int LX, int VM>
__global__ void __launch_bounds__(32 * WARPS)
k_batch_march(const BatchInst *__restrict__ insts, const BatchItem *__restrict__ items,
              int n_items, int n_steps, int step0, Barrier *bar, long long budget,
              int skip_block) {
    constexpr bool VIN = VM != V_NONE;
    using M = typename MarchOf<T, P, LX, VM, VIN>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename M::Slot *ring =
        reinterpret_cast<typename M::Slot *>(smem_raw) + (threadIdx.x >> 5) * NSLOT;
    const int lane = threadIdx.x & 31;
    if (*static_cast<volatile int *>(&bar->err)) return;
    for (int s = 0; s < n_steps; ++s) {
        // step s takes items from next[s & 1]; next[(s + 1) & 1] served step
        // s - 1, which every block has finished, and serves step s + 1, which
        // starts after the next barrier (whose fence publishes the reset)
        if (blockIdx.x == 0 && threadIdx.x == 0) bar->next[(s + 1) & 1] = 0;
        for (;;) {
            // items go to whichever warp is free next: the step ends with at
            // most one item's worth of imbalance left at the barrier
            int it = 0;
            if (lane == 0) it = int(atomicAdd(&bar->next[s & 1], 1u));
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it >= n_items) break;
            const BatchItem bi = items[it];
            const BatchInst &I = insts[bi.inst];
            const int src = (I.cur + step0 + s) & 1;
            M m;
            m.in = static_cast<const T *>(I.buf[src]);
            m.out = static_cast<T *>(I.buf[src ^ 1]);
            m.midx = I.midx;
            m.table = static_cast<const MedRec<T> *>(I.table);
            m.pitch = I.pitch;
            m.plane = I.plane;
            m.total = I.total;
            m.run_item(I.nx, I.ny, I.seg, I.n_wx, bi.item, ring);
        }
        if (!grid_barrier(bar, budget, s == 0 && int(blockIdx.x) == skip_block)) return;
    }
}

// The same for FP32 E_z batches split by plateaus: every warp takes units
// (a plateau item four columns per lane, or a two-column unit of another
// item) from the shared counter; the other items' units come first.
template <int VM>
__global__ void __launch_bounds__(32 * WARPS)
k_batch_plateau(const BatchInst *__restrict__ insts, const BatchUnit *__restrict__ units,
                int n_units, int n_steps, int step0, Barrier *bar, long long budget,
                int skip_block) {
    constexpr bool VIN = VM != V_NONE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *ring = smem_raw + (threadIdx.x >> 5) * plateau_ring_bytes<VM, VIN>();
    const int lane = threadIdx.x & 31;
    if (*static_cast<volatile int *>(&bar->err)) return;
    for (int s = 0; s < n_steps; ++s) {
        if (blockIdx.x == 0 && threadIdx.x == 0) bar->next[(s + 1) & 1] = 0;
        for (;;) {
            int it = 0;
            if (lane == 0) it = int(atomicAdd(&bar->next[s & 1], 1u));
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it >= n_units) break;
            const BatchUnit bu = units[it];
            const BatchInst &I = insts[bu.inst];
            const int src = (I.cur + step0 + s) & 1;
            run_plateau_unit<VM, VIN>(static_cast<const float *>(I.buf[src]),
                                      static_cast<float *>(I.buf[src ^ 1]), I.midx,
                                      static_cast<const MedRec<float> *>(I.table), I.nx, I.ny,
                                      I.pitch, I.plane, bu.u, ring);
        }
        if (!grid_barrier(bar, budget, s == 0 && int(blockIdx.x) == skip_block)) return;
    }
}

// Energy of every instance (as qla_energy): block (b, k) sums part b of
// instance k; the state is the buffer after `steps` steps of this run.
template <typename T, int P, int VM>
__global__ void __launch_bounds__(256)
k_batch_energy_partial(const BatchInst *__restrict__ insts, int steps,
                       double *__restrict__ partials) {
    const BatchInst &I = insts[blockIdx.y];
    const T *q = static_cast<const T *>(I.buf[(I.cur + steps) & 1]);
    const bool vin = steps > 0 ? VM != V_NONE : I.vin != 0;
    const MedRec<T> *table = static_cast<const MedRec<T> *>(I.table);
    const size_t N = size_t(I.nx) * I.ny;
    double acc = 0.0;
    for (size_t t = blockIdx.x * size_t(256) + threadIdx.x; t < N;
         t += size_t(gridDim.x) * 256) {
        const int j = int(t / I.nx), i = int(t - size_t(j) * I.nx);
        const size_t g = size_t(j) * I.pitch + i;
        T s[6];
        load_site<T, P, VM>(q, I.plane, g, vin, I.midx, table, s);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (plane_of<P>(c) < 0) continue;
            const double v = double(s[c]);
            acc = fma(v, v, acc);
        }
    }
    __shared__ double part[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += part[w];
        partials[size_t(blockIdx.y) * gridDim.x + blockIdx.x] = v;
    }
}

__global__ void k_batch_energy_final(const double *__restrict__ partials, int blocks,
                                     double *__restrict__ out) {
    if (threadIdx.x != 0) return;
    double v = 0.0;
    for (int b = 0; b < blocks; ++b) v += partials[size_t(blockIdx.x) * blocks + b];
    out[blockIdx.x] = v;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace
}  // namespace qla

using namespace qla;

struct qla_batch {
    int count = 0;
    int prec = 0, P = 6, vmode = 0;
    unsigned flags = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;     // private stream for graph capture (the
                                    // legacy default stream cannot capture)
    int device = 0, num_sms = 0;
    bool owns_ws = false;
    char *ws = nullptr;
    std::vector<qla_ctx *> inst;
    BatchInst *d_insts = nullptr;
    BatchItem *d_items = nullptr;   // the work list (BatchItem or BatchUnit entries)
    size_t items_cap = 0, units_cap = 0;
    Barrier *d_bar = nullptr;
    double *d_partials = nullptr, *d_energy = nullptr;
    int lane_cols = 0, rows = 0;
    long long budget = 1LL << 31;
    int skip_block = -1;
    long long launches = 0;
    std::string err;
};

namespace {

qla_status bfail(qla_batch *b, qla_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return s;
}

#define BCUDA(b, call, what)                                                     \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess)                                                   \
            return bfail((b), QLA_ECUDA, "%s: %s", (what), cudaGetErrorString(e_)); \
    } while (0)

bool lattice_ok(int nx, int ny, int planes) {
    return nx >= 128 && nx % 4 == 0 && ny >= 8 &&
           offsets32_ok(size_t(planes), padded_plane(nx, ny));
}

// Work-list capacity (rows per item >= 32): items of the two-column
// layout, or units of the plateau split (three per 120-column item).
size_t items_of(int count, const int *nx, const int *ny) {
    size_t items = 0;
    for (int k = 0; k < count; ++k)
        items += size_t((nx[k] + 55) / 56) * size_t((ny[k] + 31) / 32);
    return items;
}
size_t units_of(int count, const int *nx, const int *ny) {
    size_t units = 0;
    for (int k = 0; k < count; ++k)
        units += 3 * size_t((nx[k] + PWOUT - 1) / PWOUT) * size_t((ny[k] + 31) / 32);
    return units;
}
size_t list_bytes(int count, const int *nx, const int *ny) {
    return std::max(sizeof(BatchItem) * items_of(count, nx, ny),
                    sizeof(BatchUnit) * units_of(count, nx, ny));
}

size_t tail_bytes(int count, const int *nx, const int *ny) {
    size_t t = 0;
    t += align256(sizeof(BatchInst) * count);
    t += align256(list_bytes(count, nx, ny));
    t += align256(sizeof(Barrier));
    t += align256(sizeof(double) * count * ENERGY_BLOCKS);
    t += align256(sizeof(double) * count * ENERGY_ROWS);
    return t;
}

// Kernel set for the batch's precision / planes / lane width / V reading.
struct Kern {
    const void *march;
    size_t slot_bytes;
    const void *epart;
    bool plateau;   // the plateau-split kernel (units instead of items)
};

template <typename T, int P, int LX, int VM>
Kern kern_t() {
    if constexpr (std::is_same<T, float>::value && P == 3 && LX == 2) {
        // FP32 E_z, two columns per lane: split by plateaus
        return Kern{reinterpret_cast<const void *>(&k_batch_plateau<VM>),
                    plateau_ring_bytes<VM, VM != V_NONE>() / NSLOT,
                    reinterpret_cast<const void *>(&k_batch_energy_partial<T, P, VM>), true};
    } else {
        using M = typename MarchOf<T, P, LX, VM, VM != V_NONE>::type;
        return Kern{reinterpret_cast<const void *>(&k_batch_march<T, P, LX, VM>),
                    sizeof(typename M::Slot),
                    reinterpret_cast<const void *>(&k_batch_energy_partial<T, P, VM>), false};
    }
}

template <typename T, int P, int LX>
Kern kern_vm(int vm) {
    return vm == V_ROTATION ? kern_t<T, P, LX, V_ROTATION>()
         : vm == V_LITERAL  ? kern_t<T, P, LX, V_LITERAL>()
                            : kern_t<T, P, LX, V_NONE>();
}

Kern kernels(const qla_batch *b, int lx) {
    if (b->prec == QLA_FP64)
        return b->P == 6 ? kern_vm<double, 6, 2>(b->vmode) : kern_vm<double, 3, 2>(b->vmode);
    if (b->P == 6) return kern_vm<float, 6, 2>(b->vmode);
    return lx == 4 ? kern_vm<float, 3, 4>(b->vmode)
         : lx == 1 ? kern_vm<float, 3, 1>(b->vmode)
                   : kern_vm<float, 3, 2>(b->vmode);
}

// FP32 E_z batches: packed pairs (1), 2 (the default) or 4 adjacent columns
// per lane; other batches: 2.
int lane_cols_of(const qla_batch *b) {
    if (b->prec == QLA_FP32 && b->P == 3) return b->lane_cols == 0 ? 2 : b->lane_cols;
    return 2;
}

int window_out(int lx) { return lx == 1 ? 56 : 32 * lx - 8; }

// Interleave per-instance lists so that each wave mixes lattices.
template <typename E>
void interleave(const std::vector<std::vector<E>> &per, std::vector<E> &out) {
    std::vector<size_t> pos(per.size(), 0);
    for (bool any = true; any;) {
        any = false;
        for (size_t k = 0; k < per.size(); ++k)
            if (pos[k] < per[k].size()) {
                out.push_back(per[k][pos[k]++]);
                any = true;
            }
    }
}

// Units of the plateau-split kernel (segments of `seg` rows, capped at each
// lattice's height): every instance's items classified on the GPU (into the
// batch's work list, which the units then replace; the instances' own unit
// lists belong to their single-lattice steps), then the other items' units
// of all instances, interleaved, followed by the plateau units, interleaved.
qla_status build_units(qla_batch *b, int rows, int *n_units, std::vector<BatchInst> &hinst) {
    std::vector<int> segs(b->count), nwx(b->count), nitems(b->count);
    std::vector<size_t> at(b->count + 1, 0);
    for (int k = 0; k < b->count; ++k) {
        qla_ctx *c = b->inst[k];
        // 128-row segments by default (256 instances of sides 512-2048:
        // 1.64e11 site-updates/s at 64 or 128 rows, 1.52e11 at 256)
        int seg = rows > 0 ? rows : 128;
        seg = (seg + 3) / 4 * 4;
        if (seg > c->ny) seg = (c->ny + 3) / 4 * 4;
        segs[k] = seg;
        nwx[k] = (c->nx + PWOUT - 1) / PWOUT;
        nitems[k] = nwx[k] * ((c->ny + seg - 1) / seg);
        at[k + 1] = at[k] + size_t(nitems[k]);
    }
    if (at[b->count] > b->units_cap)   // classes take 4 of a unit's 32 bytes
        return bfail(b, QLA_EINVAL, "qla_batch: %zu items exceed the workspace's %zu",
                     at[b->count], b->units_cap);
    int *cls_dev = reinterpret_cast<int *>(b->d_items);
    for (int k = 0; k < b->count; ++k) {
        qla_ctx *c = b->inst[k];
        k_classify_items<<<(nitems[k] + WARPS - 1) / WARPS, 32 * WARPS, 0, b->stream>>>(
            c->midx, c->nx, c->ny, c->pitch, segs[k], nwx[k], nitems[k], cls_dev + at[k]);
        BCUDA(b, cudaGetLastError(), "qla_batch: classify");
    }
    std::vector<int> all(at[b->count]);
    BCUDA(b, cudaMemcpyAsync(all.data(), cls_dev, all.size() * 4, cudaMemcpyDeviceToHost,
                             b->stream), "qla_batch: classes");
    BCUDA(b, cudaStreamSynchronize(b->stream), "qla_batch: classes");
    std::vector<std::vector<int>> cls(b->count);
    for (int k = 0; k < b->count; ++k)
        cls[k].assign(all.begin() + at[k], all.begin() + at[k + 1]);
    std::vector<std::vector<BatchUnit>> other(b->count), plat(b->count);
    for (int k = 0; k < b->count; ++k) {
        qla_ctx *c = b->inst[k];
        std::vector<int4> o, p;
        plateau_units(cls[k], c->nx, c->ny, segs[k], o, p);
        for (const int4 &u : o) other[k].push_back(BatchUnit{u, k, 0, 0, 0});
        for (const int4 &u : p) plat[k].push_back(BatchUnit{u, k, 0, 0, 0});
    }
    std::vector<BatchUnit> list;
    interleave(other, list);
    interleave(plat, list);
    if (list.size() > b->units_cap)
        return bfail(b, QLA_EINVAL, "qla_batch: %zu units exceed the workspace's %zu",
                     list.size(), b->units_cap);
    BCUDA(b, cudaMemcpyAsync(b->d_items, list.data(), list.size() * sizeof(BatchUnit),
                             cudaMemcpyHostToDevice, b->stream), "qla_batch: units");
    hinst.resize(b->count);
    for (int k = 0; k < b->count; ++k) {
        qla_ctx *c = b->inst[k];
        BatchInst &I = hinst[k];
        I.buf[0] = c->state[0];
        I.buf[1] = c->state[1];
        I.midx = c->midx;
        I.table = c->table;
        I.nx = c->nx;
        I.ny = c->ny;
        I.pitch = c->pitch;
        I.seg = segs[k];
        I.n_wx = nwx[k];
        I.plane = uint32_t(c->plane_elems);
        I.total = uint32_t(c->ny) * uint32_t(c->pitch);
        I.cur = c->cur;
        I.vin = c->pending_v ? 1 : 0;
    }
    BCUDA(b, cudaMemcpyAsync(b->d_insts, hinst.data(), hinst.size() * sizeof(BatchInst),
                             cudaMemcpyHostToDevice, b->stream), "qla_batch: instances");
    BCUDA(b, cudaStreamSynchronize(b->stream), "qla_batch: upload");
    *n_units = int(list.size());
    return QLA_OK;
}

// Work items for the current tiling; returns the item count.
qla_status build_items(qla_batch *b, int lx, int rows, int *n_items,
                       std::vector<BatchInst> &hinst) {
    if (kernels(b, lx).plateau) return build_units(b, rows, n_items, hinst);
    const int wout = window_out(lx);
    std::vector<BatchItem> items;
    hinst.resize(b->count);
    for (int k = 0; k < b->count; ++k) {
        qla_ctx *c = b->inst[k];
        int seg = rows > 0 ? rows : 256;
        seg = (seg + 3) / 4 * 4;
        if (seg > c->ny) seg = (c->ny + 3) / 4 * 4;
        const int n_wx = (c->nx + wout - 1) / wout, n_wy = (c->ny + seg - 1) / seg;
        BatchInst &I = hinst[k];
        I.buf[0] = c->state[0];
        I.buf[1] = c->state[1];
        I.midx = c->midx;
        I.table = c->table;
        I.nx = c->nx;
        I.ny = c->ny;
        I.pitch = c->pitch;
        I.seg = seg;
        I.n_wx = n_wx;
        I.plane = uint32_t(c->plane_elems);
        I.total = uint32_t(c->ny) * uint32_t(c->pitch);
        I.cur = c->cur;
        I.vin = c->pending_v ? 1 : 0;
        for (int i = 0; i < n_wx * n_wy; ++i) items.push_back(BatchItem{k, i});
    }
    // interleave instances so that each wave mixes lattices
    std::vector<BatchItem> mixed;
    mixed.reserve(items.size());
    {
        std::vector<size_t> start(b->count + 1, 0), pos(b->count, 0);
        for (const BatchItem &it : items) start[it.inst + 1]++;
        for (int k = 0; k < b->count; ++k) start[k + 1] += start[k];
        bool any = true;
        while (any) {
            any = false;
            for (int k = 0; k < b->count; ++k) {
                if (start[k] + pos[k] < start[k + 1]) {
                    mixed.push_back(items[start[k] + pos[k]++]);
                    any = true;
                }
            }
        }
    }
    if (mixed.size() > b->items_cap)
        return bfail(b, QLA_EINVAL, "qla_batch: %zu work items exceed the workspace's %zu "
                     "(rows per item below 32?)", mixed.size(), b->items_cap);
    BCUDA(b, cudaMemcpyAsync(b->d_items, mixed.data(), mixed.size() * sizeof(BatchItem),
                             cudaMemcpyHostToDevice, b->stream), "qla_batch: items");
    BCUDA(b, cudaMemcpyAsync(b->d_insts, hinst.data(), hinst.size() * sizeof(BatchInst),
                             cudaMemcpyHostToDevice, b->stream), "qla_batch: instances");
    BCUDA(b, cudaStreamSynchronize(b->stream), "qla_batch: upload");
    *n_items = int(mixed.size());
    return QLA_OK;
}

// Grid of the persistent kernel: every block co-resident.
qla_status grid_for(qla_batch *b, const Kern &k, int *blocks, size_t *smem) {
    *smem = k.slot_bytes * NSLOT * WARPS;
    BCUDA(b, cudaFuncSetAttribute(k.march, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(*smem)), "qla_batch: smem attribute");
    int per_sm = 0;
    BCUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.march, 32 * WARPS, *smem),
          "qla_batch: occupancy");
    if (per_sm < 1) return bfail(b, QLA_ECUDA, "qla_batch: kernel does not fit an SM");
    *blocks = per_sm * b->num_sms;
    return QLA_OK;
}

qla_status launch_chunk(qla_batch *b, cudaStream_t st, const Kern &k, int blocks, size_t smem,
                        int n_items, int n_steps, int step0) {
    BCUDA(b, cudaMemsetAsync(b->d_bar, 0, offsetof(Barrier, err), st),
          "qla_batch: barrier reset");
    void *args[] = {&b->d_insts, &b->d_items, &n_items, &n_steps, &step0, &b->d_bar,
                    &b->budget, &b->skip_block};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(32 * WARPS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BCUDA(b, cudaLaunchKernelExC(&cfg, k.march, args), "qla_batch: persistent launch");
    b->launches++;
    return QLA_OK;
}

qla_status launch_energy(qla_batch *b, cudaStream_t st, const Kern &k, int steps, double *out) {
    void *args[] = {&b->d_insts, &steps, &b->d_partials};
    BCUDA(b, cudaLaunchKernel(k.epart, dim3(ENERGY_BLOCKS, b->count), dim3(256), args, 0, st),
          "qla_batch: energy");
    k_batch_energy_final<<<b->count, 32, 0, st>>>(b->d_partials, ENERGY_BLOCKS, out);
    BCUDA(b, cudaGetLastError(), "qla_batch: energy final");
    b->launches += 2;
    return QLA_OK;
}

// Bring every instance to "potential operator pending" with one ordinary
// step if any is not (the persistent kernel always applies the pending V).
qla_status align_pending(qla_batch *b, long long *n_steps) {
    if (b->vmode == V_NONE || *n_steps == 0) return QLA_OK;
    bool all = true;
    for (qla_ctx *c : b->inst) all = all && c->pending_v;
    if (all) return QLA_OK;
    for (qla_ctx *c : b->inst) {
        const qla_status s = qla_step(c, 1);
        if (s != QLA_OK) return bfail(b, s, "qla_batch: first step: %s", qla_last_error(c));
    }
    --*n_steps;
    return QLA_OK;
}

qla_status check_ready(qla_batch *b) {
    for (int k = 0; k < b->count; ++k) {
        qla_ctx *c = b->inst[k];
        if (c->sticky != QLA_OK) return bfail(b, c->sticky, "instance %d is unusable", k);
        if (!c->has_medium || !c->has_state)
            return bfail(b, QLA_ESTATE, "instance %d has no medium or state", k);
    }
    return QLA_OK;
}

void finish(qla_batch *b, long long steps) {
    for (qla_ctx *c : b->inst) {
        c->cur = (c->cur + int(steps & 1)) & 1;
        if (steps > 0 && c->vmode != V_NONE) c->pending_v = true;
    }
}

qla_status read_err(qla_batch *b) {
    int e = 0;
    BCUDA(b, cudaMemcpyAsync(&e, &b->d_bar->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
          "qla_batch: error word");
    BCUDA(b, cudaStreamSynchronize(b->stream), "qla_batch: sync");
    if (e) return bfail(b, QLA_ETIMEOUT, "qla_batch: a grid barrier wait ran out");
    return QLA_OK;
}

// Step all instances n_steps (after align_pending); no synchronisation.
// e0 (if given) is recorded on the stream once the work list is built, so
// that a timing around the call sees the launches only.
qla_status step_persistent(qla_batch *b, long long n_steps, int lx, int rows,
                           cudaEvent_t e0 = nullptr) {
    std::vector<BatchInst> hinst;
    int n_items = 0;
    qla_status s = build_items(b, lx, rows, &n_items, hinst);
    if (s != QLA_OK) return s;
    const Kern k = kernels(b, lx);
    int blocks = 0;
    size_t smem = 0;
    s = grid_for(b, k, &blocks, &smem);
    if (s != QLA_OK) return s;
    if (e0) BCUDA(b, cudaEventRecord(e0, b->stream), "qla_batch: event");
    for (long long done = 0; done < n_steps;) {
        const int chunk = int(std::min<long long>(QLA_BATCH_CHUNK, n_steps - done));
        s = launch_chunk(b, b->stream, k, blocks, smem, n_items, chunk, int(done & 1));
        if (s != QLA_OK) return s;
        done += chunk;
    }
    finish(b, n_steps);
    return QLA_OK;
}

}  // namespace

extern "C" {

size_t qla_batch_workspace_bytes(int count, const int *nx, const int *ny, int precision,
                                 unsigned flags) {
    if (count < 1 || !nx || !ny) return 0;
    if (flags & (QLA_ANISOTROPIC | QLA_POTENTIAL_LCU)) return 0;  // single contexts only
    size_t total = 0;
    for (int k = 0; k < count; ++k) {
        if (!lattice_ok(nx[k], ny[k], (flags & QLA_TE_ONLY) ? 3 : 6)) return 0;
        const size_t b = qla_workspace_bytes(nx[k], ny[k], precision, flags);
        if (b == 0) return 0;
        total += align256(b);
    }
    return total + tail_bytes(count, nx, ny);
}

qla_status qla_batch_create(qla_batch **out, int count, const int *nx, const int *ny,
                            double delta, int precision, unsigned flags, void *cuda_stream,
                            void *workspace, size_t workspace_bytes) {
    if (!out) return QLA_EINVAL;
    *out = nullptr;
    const size_t need = qla_batch_workspace_bytes(count, nx, ny, precision, flags);
    if (need == 0) return QLA_EINVAL;
    if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255)) return QLA_EINVAL;
    if (workspace && workspace_bytes < need) return QLA_ENOMEM;
    qla_batch *b = new (std::nothrow) qla_batch();
    if (!b) return QLA_ENOMEM;
    b->count = count;
    b->prec = precision;
    b->flags = flags;
    b->P = (flags & QLA_TE_ONLY) ? 3 : 6;
    b->vmode = (flags & QLA_POTENTIAL_LITERAL) ? V_LITERAL
             : (flags & QLA_POTENTIAL_NONE)    ? V_NONE
                                               : V_ROTATION;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&b->device) != cudaSuccess) { delete b; return QLA_ECUDA; }
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return QLA_ECUDA;
    }
    if (workspace) {
        b->ws = static_cast<char *>(workspace);
    } else {
        void *p = nullptr;
        if (cudaMalloc(&p, need) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return QLA_ENOMEM;
        }
        b->ws = static_cast<char *>(p);
        b->owns_ws = true;
    }
    size_t off = 0;
    b->inst.assign(count, nullptr);
    for (int k = 0; k < count; ++k) {
        const size_t sz = qla_workspace_bytes(nx[k], ny[k], precision, flags);
        const qla_status s = qla_init_grid(&b->inst[k], nx[k], ny[k], delta, precision, flags,
                                           cuda_stream, b->ws + off, sz);
        if (s != QLA_OK) {
            qla_batch_destroy(b);
            return s;
        }
        off += align256(sz);
    }
    b->d_insts = reinterpret_cast<BatchInst *>(b->ws + off);
    off += align256(sizeof(BatchInst) * count);
    b->d_items = reinterpret_cast<BatchItem *>(b->ws + off);
    b->items_cap = items_of(count, nx, ny);
    b->units_cap = units_of(count, nx, ny);
    off += align256(list_bytes(count, nx, ny));
    b->d_bar = reinterpret_cast<Barrier *>(b->ws + off);
    off += align256(sizeof(Barrier));
    b->d_partials = reinterpret_cast<double *>(b->ws + off);
    off += align256(sizeof(double) * count * ENERGY_BLOCKS);
    b->d_energy = reinterpret_cast<double *>(b->ws + off);
    if (cudaMemsetAsync(b->d_bar, 0, sizeof(Barrier), b->stream) != cudaSuccess) {
        qla_batch_destroy(b);
        return QLA_ECUDA;
    }
    *out = b;
    return QLA_OK;
}

qla_ctx *qla_batch_instance(qla_batch *b, int k) {
    if (!b || k < 0 || k >= b->count) return nullptr;
    return b->inst[k];
}

qla_status qla_batch_set_tuning(qla_batch *b, int lane_cols, int rows) {
    if (!b) return QLA_EINVAL;
    if (lane_cols != 0 && lane_cols != 1 && lane_cols != 2 && lane_cols != 4)
        return bfail(b, QLA_EINVAL, "qla_batch_set_tuning: lane_cols %d", lane_cols);
    if (rows != 0 && (rows < 32 || rows > (1 << 20)))
        return bfail(b, QLA_EINVAL, "qla_batch_set_tuning: rows %d (0 or >= 32)", rows);
    b->lane_cols = lane_cols;
    b->rows = rows;
    return QLA_OK;
}

qla_status qla_batch_debug_barrier(qla_batch *b, long long budget_cycles, int skip_block) {
    if (!b) return QLA_EINVAL;
    b->budget = budget_cycles > 0 ? budget_cycles : (1LL << 31);
    b->skip_block = skip_block;
    return QLA_OK;
}

qla_status qla_batch_step(qla_batch *b, long long n_steps) {
    if (!b) return QLA_EINVAL;
    if (n_steps < 0) return bfail(b, QLA_EINVAL, "qla_batch_step: n_steps < 0");
    qla_status s = check_ready(b);
    if (s != QLA_OK || n_steps == 0) return s;
    BCUDA(b, cudaMemsetAsync(b->d_bar, 0, sizeof(Barrier), b->stream), "qla_batch: reset");
    s = align_pending(b, &n_steps);
    if (s != QLA_OK) return s;
    s = step_persistent(b, n_steps, lane_cols_of(b), b->rows);
    if (s != QLA_OK) return s;
    return read_err(b);
}

qla_status qla_batch_energy(qla_batch *b, double *out) {
    if (!b || !out) return QLA_EINVAL;
    for (int k = 0; k < b->count; ++k) {
        const qla_status s = qla_energy(b->inst[k], out + k);
        if (s != QLA_OK) return bfail(b, s, "instance %d: %s", k, qla_last_error(b->inst[k]));
    }
    return QLA_OK;
}

qla_status qla_batch_run(qla_batch *b, long long n_steps, long long every, double *energies) {
    if (!b || !energies) return QLA_EINVAL;
    if (every < 1 || n_steps < 0 || n_steps % every)
        return bfail(b, QLA_EINVAL, "qla_batch_run: n_steps must be a multiple of every >= 1");
    qla_status s = check_ready(b);
    if (s != QLA_OK || n_steps == 0) return s;
    BCUDA(b, cudaMemsetAsync(b->d_bar, 0, sizeof(Barrier), b->stream), "qla_batch: reset");
    // the first step of the run may need the ordinary kernel (see
    // align_pending); it then belongs to the first energy interval
    long long first = 0;
    {
        long long n = n_steps;
        s = align_pending(b, &n);
        if (s != QLA_OK) return s;
        first = n_steps - n;
    }
    const int lx = lane_cols_of(b);
    std::vector<BatchInst> hinst;
    int n_items = 0;
    s = build_items(b, lx, b->rows, &n_items, hinst);
    if (s != QLA_OK) return s;
    const Kern k = kernels(b, lx);
    int blocks = 0;
    size_t smem = 0;
    s = grid_for(b, k, &blocks, &smem);
    if (s != QLA_OK) return s;
    const long long rows_total = n_steps / every;
    long long done = 0;  // persistent steps since hinst was built
    for (long long r0 = 0; r0 < rows_total; r0 += ENERGY_ROWS) {
        const int nrows = int(std::min<long long>(ENERGY_ROWS, rows_total - r0));
        // capture nrows x (steps, energy) as one graph and replay it once
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        BCUDA(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal),
              "qla_batch_run: capture");
        qla_status cs = QLA_OK;
        long long d = done;
        for (int r = 0; r < nrows && cs == QLA_OK; ++r) {
            long long steps = every - ((r0 + r) == 0 ? first : 0);
            for (long long x = 0; x < steps && cs == QLA_OK;) {
                const int chunk = int(std::min<long long>(QLA_BATCH_CHUNK, steps - x));
                cs = launch_chunk(b, b->cap, k, blocks, smem, n_items, chunk, int(d & 1));
                x += chunk;
                d += chunk;
            }
            // the energy kernel needs only the parity of d and whether d > 0
            if (cs == QLA_OK)
                cs = launch_energy(b, b->cap, k, int((d & 1) + (d > 0 ? 2 : 0)),
                                   b->d_energy + size_t(r) * b->count);
        }
        cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
        if (cs != QLA_OK) {
            if (graph) cudaGraphDestroy(graph);
            return cs;
        }
        BCUDA(b, ce, "qla_batch_run: end capture");
        ce = cudaGraphInstantiate(&exec, graph, 0);
        if (ce != cudaSuccess) {
            cudaGraphDestroy(graph);
            return bfail(b, QLA_ECUDA, "qla_batch_run: instantiate: %s", cudaGetErrorString(ce));
        }
        ce = cudaGraphLaunch(exec, b->stream);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(energies + size_t(r0) * b->count, b->d_energy,
                                 sizeof(double) * nrows * b->count, cudaMemcpyDeviceToHost,
                                 b->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        BCUDA(b, ce, "qla_batch_run: replay");
        done = d;
        b->launches++;
    }
    finish(b, done);
    return read_err(b);
}

qla_status qla_batch_autotune(qla_batch *b, int trial_steps, int *chosen_lane_cols,
                              int *chosen_rows) {
    if (!b || trial_steps < 1) return QLA_EINVAL;
    qla_status s = check_ready(b);
    if (s != QLA_OK) return s;
    long long n = 6LL * trial_steps;
    BCUDA(b, cudaMemsetAsync(b->d_bar, 0, sizeof(Barrier), b->stream), "qla_batch: reset");
    s = align_pending(b, &n);
    if (s != QLA_OK) return s;
    const bool two = b->prec == QLA_FP32 && b->P == 3;
    const int lxs[2] = {1, 2};
    const int rowss[3] = {64, 128, 256};
    float best = 1e30f;
    int best_lx = 2, best_rows = 256;
    cudaEvent_t e0, e1;
    BCUDA(b, cudaEventCreate(&e0), "qla_batch_autotune: event");
    BCUDA(b, cudaEventCreate(&e1), "qla_batch_autotune: event");
    long long used = 6LL * trial_steps - n;  // steps already taken by align_pending
    for (int li = 0; li < 2; ++li) {
        for (int ri = 0; ri < 3; ++ri) {
            const int lx = two ? lxs[li] : 2;
            long long steps = trial_steps - (li == 0 && ri == 0 ? used : 0);
            if (steps <= 0) steps = 1;
            s = step_persistent(b, steps, lx, rowss[ri], e0);
            cudaEventRecord(e1, b->stream);
            if (s != QLA_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) { s = QLA_ECUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= float(steps);
            if (ms < best) {
                best = ms;
                best_lx = lx;
                best_rows = rowss[ri];
            }
        }
        if (s != QLA_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != QLA_OK) return s;
    s = read_err(b);
    if (s != QLA_OK) return s;
    b->lane_cols = best_lx;
    b->rows = best_rows;
    if (chosen_lane_cols) *chosen_lane_cols = best_lx;
    if (chosen_rows) *chosen_rows = best_rows;
    return QLA_OK;
}

long long qla_batch_launch_count(const qla_batch *b) { return b ? b->launches : 0; }

const char *qla_batch_last_error(const qla_batch *b) { return b ? b->err.c_str() : "null batch"; }

void qla_batch_destroy(qla_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    for (qla_ctx *c : b->inst)
        if (c) qla_destroy(c);
    if (b->owns_ws) cudaFree(b->ws);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaGetLastError();
    delete b;
}

}  // extern "C"
