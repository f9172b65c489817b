// Plateau work units of the E_z marching steps: FP32 (single lattices and
// batches) and double-single.
//
// In the workloads' media most sites sit on plateaus of n on which every
// site's four neighbours carry its n: those share one record (see MedRec),
// their potential step is the identity and their collision coefficients
// are the same everywhere on the plateau.  A work item whose entering sites
// all share one record -- a plateau item -- therefore needs no index rows,
// no record lookups and no potential step; without the record ring the
// march holds four columns per lane (128-column windows, 8 of 128 columns
// recomputed instead of 8 of 64) in the register budget of the two-column
// march.  Every other item runs the two-column march with its record ring.
//
// A unit is one warp's work: int4 (x_out, w_out | (rec + 1) << 8, y_lo,
// y_hi) = store columns [x_out, x_out + w_out) of rows [y_lo, y_hi); rec is
// the plateau record (>= 0: the four-column plateau march with that
// record's coefficients) or -1 (the two-column march, w_out <= 56).
// w_out = 0 marks an idle warp.
#pragma once

#include <algorithm>
#include <vector>

#include "qla_march.cuh"

namespace qla {
namespace march {

constexpr int PW = 128, PWOUT = 120;   // plateau windows: columns, stored columns
constexpr int GWOUT = 56;              // stored columns of a two-column window

__host__ __device__ inline int4 plateau_unit(int x_out, int w_out, int rec, int y_lo, int y_hi) {
    return make_int4(x_out, w_out | ((rec + 1) << 8), y_lo, y_hi);
}

// Run unit u of a lattice (arrays in/out/midx/table of its size and pitch);
// smem: this warp's staging ring (room for the four-column ring).
template <int VM, bool VIN>
__device__ __forceinline__ void run_plateau_unit(const float *in, float *out, const uint32_t *midx,
                                                 const MedRec<float> *table, int nx, int ny,
                                                 int pitch, uint32_t plane, const int4 &u,
                                                 unsigned char *smem) {
    const int w_out = u.y & 0xff, rec = (u.y >> 8) - 1;
    if (w_out == 0) return;
    if (rec >= 0) {
        using M = March<float, 3, 4, VM, VIN, true>;
        M m;
        m.in = in;
        m.out = out;
        m.midx = midx;
        m.table = table;
        m.pitch = pitch;
        m.plane = plane;
        m.total = uint32_t(ny) * uint32_t(pitch);
        // the same 16 bytes in every lane
        m.set_uniform(__ldg(&table[rec].c));
        m.run_unit(nx, ny, u.x, w_out, u.z, u.w, reinterpret_cast<typename M::Slot *>(smem));
    } else {
        using M = March<float, 3, 2, VM, VIN, false>;
        M m;
        m.in = in;
        m.out = out;
        m.midx = midx;
        m.table = table;
        m.pitch = pitch;
        m.plane = plane;
        m.total = uint32_t(ny) * uint32_t(pitch);
        m.run_unit(nx, ny, u.x, w_out, u.z, u.w, reinterpret_cast<typename M::Slot *>(smem));
    }
}

// The same for double-single steps (FP64 state in word pairs): both kinds
// of unit are 64-column windows (two columns per lane); a plateau unit
// drops the record ring -- 64 registers of three-word coefficients -- and
// takes its record's coefficients once.
template <int VM, bool VIN>
__device__ __forceinline__ void run_ds_unit(const dsf *in, dsf *out, const uint32_t *midx,
                                            const MedRec<dsf> *table, int nx, int ny, int pitch,
                                            uint32_t plane, const int4 &u, unsigned char *smem) {
    const int w_out = u.y & 0xff, rec = (u.y >> 8) - 1;
    if (w_out == 0) return;
    if (rec >= 0) {
        using M = March<dsf, 3, 2, VM, VIN, true>;
        M m;
        m.in = in;
        m.out = out;
        m.midx = midx;
        m.table = table;
        m.pitch = pitch;
        m.plane = plane;
        m.total = uint32_t(ny) * uint32_t(pitch);
        m.set_uniform(table[rec].c);   // the same 32 bytes in every lane
        m.run_unit(nx, ny, u.x, w_out, u.z, u.w, reinterpret_cast<typename M::Slot *>(smem));
    } else {
        using M = March<dsf, 3, 2, VM, VIN, false>;
        M m;
        m.in = in;
        m.out = out;
        m.midx = midx;
        m.table = table;
        m.pitch = pitch;
        m.plane = plane;
        m.total = uint32_t(ny) * uint32_t(pitch);
        m.run_unit(nx, ny, u.x, w_out, u.z, u.w, reinterpret_cast<typename M::Slot *>(smem));
    }
}

// Bytes of one warp's staging ring for either march.
template <int VM, bool VIN> constexpr size_t plateau_ring_bytes() {
    return std::max(sizeof(typename March<float, 3, 4, VM, VIN, true>::Slot),
                    sizeof(typename March<float, 3, 2, VM, VIN, false>::Slot)) *
           NSLOT;
}

namespace {

// The record shared by all entering sites of each item of a window layout
// (CPL columns per lane: columns [x0, x0 + 32 CPL) and rows [y_lo - 4,
// y_hi + 4), periodic, with x0 = (32 CPL - 8) wx - 4), or -1 where they
// differ or the record is a site's own: one warp per item.  CPL = 4: the
// plateau windows of FP32 E_z steps; 2: the 64-column windows of
// double-single steps.
template <int CPL>
__global__ void k_classify(const uint32_t *__restrict__ midx, int nx, int ny, int pitch,
                           int seg_h, int n_wx, int n_items, int *__restrict__ cls) {
    const int item = int(blockIdx.x) * WARPS + int(threadIdx.x >> 5);
    if (item >= n_items) return;   // the whole warp
    const int lane = threadIdx.x & 31;
    const int wx = item % n_wx, wy = item / n_wx;
    const int x0 = wx * (32 * CPL - 8) - 4 + CPL * lane;
    int col[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) col[k] = wrap(x0 + k, nx);
    const int y_lo = wy * seg_h, y_hi = min(ny, y_lo + seg_h);
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (int J = y_lo - LAG; J < y_hi + LAG; ++J) {
        const uint32_t *row = midx + size_t(wrap(J, ny)) * size_t(pitch);
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const uint32_t v = __ldg(row + col[k]);
            lo = min(lo, v);
            hi = max(hi, v);
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) cls[item] = lo == hi && lo < uint32_t(UNIFORM_SLOTS) ? int(lo) : -1;
}
constexpr auto k_classify_items = k_classify<4>;

}  // namespace

// The units of one lattice from its item classes (n_wx plateau windows per
// row of items, segments of seg rows): every plateau item as one unit, every
// other item as two-column units of at most 56 columns.  Appends the other
// units to `other` and the plateau units to `plat`; returns the number of
// plateau items.
inline int plateau_units(const std::vector<int> &cls, int nx, int ny, int seg,
                         std::vector<int4> &other, std::vector<int4> &plat) {
    const int n_wx = (nx + PWOUT - 1) / PWOUT;
    int n_plateau = 0;
    for (size_t i = 0; i < cls.size(); ++i) {
        const int wx = int(i) % n_wx, wy = int(i) / n_wx;
        const int x_out = wx * PWOUT, w_out = std::min(PWOUT, nx - x_out);
        const int y_lo = wy * seg, y_hi = std::min(ny, y_lo + seg);
        if (cls[i] >= 0) {
            plat.push_back(plateau_unit(x_out, w_out, cls[i], y_lo, y_hi));
            ++n_plateau;
        } else {
            for (int x = x_out; x < x_out + w_out; x += GWOUT)
                other.push_back(plateau_unit(x, std::min(GWOUT, x_out + w_out - x), -1, y_lo, y_hi));
        }
    }
    return n_plateau;
}

// ---------------------------------------------------------------------------
// Dataflow steps: several steps of the unit list in one persistent launch.
//
// Between two steps the only ordering the step needs is local: a unit of
// step s reads its window of the buffer step s - 1 wrote (four columns and
// four rows beyond what it stores, Eqs. 2e6 and 2e9) and writes the buffer
// that step s - 1 read.  So instead of a launch (a grid-wide barrier) per
// step, warps take units of all steps from one counter in step order, and a
// unit of step s first waits until every item it depends on has finished
// step s - 1: those whose stored columns and rows it reads (read after
// write) and those that read what it stores (write after read).  Dependencies
// are always handed out earlier than their dependants, and the warp holding
// the earliest unfinished unit never waits, so the launch cannot deadlock
// whatever the residency; the warps that finish a step early start on the
// next one instead of idling at the step's tail.
//
// Per item a counter grows by 6 per finished step: a plateau unit adds 6,
// each of the n two-column units of another item 6 / n (n <= 3).  Step
// s - 1 of an item is complete when its counter reaches 6 s, since its
// step-s units wait for that themselves.

constexpr int FLOW_DEPS = 8;   // per axis: a count and up to seven indices

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait (the whole warp) until every item of the x-dependencies of window wx
// times the y-dependencies of segment wy has a counter >= target.  Each lane
// polls one dependency with an acquire load, so its later reads see what
// those items stored.  Gives up after `budget` SM cycles (raising *err) or
// when another warp has raised it; returns false then.
__device__ __forceinline__ bool flow_wait(const int *__restrict__ xdep,
                                          const int *__restrict__ ydep, const unsigned *done,
                                          int n_wx, int wx, int wy, unsigned target, int *err,
                                          long long budget) {
    const int lane = threadIdx.x & 31;
    const int cx = xdep[wx * FLOW_DEPS], cy = ydep[wy * FLOW_DEPS];
    const int n = cx * cy;
    const long long t0 = clock64();
    for (int base = 0; base < n; base += 32) {
        const int k = base + lane < n ? base + lane : base;
        const int d = ydep[wy * FLOW_DEPS + 1 + k / cx] * n_wx + xdep[wx * FLOW_DEPS + 1 + k % cx];
        for (;;) {
            const bool ok = ld_acquire_gpu(done + d) >= target;
            if (__all_sync(0xffffffffu, ok)) break;
            // decided by a vote, so that the warp leaves together
            const bool stop = *static_cast<volatile int *>(err) != 0 || clock64() - t0 > budget;
            if (__any_sync(0xffffffffu, stop)) {
                if (lane == 0) atomicExch(err, 1);
                return false;
            }
            __nanosleep(256);
        }
    }
    return true;
}

// The counter increment of unit u (window wx of a lattice nx wide).
__host__ __device__ inline unsigned flow_increment(const int4 &u, int nx, int wx) {
    if ((u.y >> 8) - 1 >= 0) return 6u;
    const int rest = nx - wx * PWOUT, w = rest < PWOUT ? rest : PWOUT;
    return 6u / unsigned((w + GWOUT - 1) / GWOUT);
}

// Host: the dependency table of one axis.  Block a of n_blocks stores
// [a * width, min(len, (a + 1) * width)) of a periodic axis of length len
// and reads [a * width - lo, read_end(a)).  Entry a * FLOW_DEPS holds the
// count, then the blocks b (a itself included) for which a's reads meet b's
// stores or b's reads meet a's stores.  Blocks more than three apart never
// do: reads reach at most 172 columns past a window's start (120-column
// windows) or four rows past a segment (at least 16 rows), and only the last
// block is narrower.  Returns false if a block has more than seven.
template <typename ReadEnd>
inline bool flow_axis_deps(long long len, int width, int n_blocks, int lo, ReadEnd read_end,
                           std::vector<int> &out) {
    out.assign(size_t(n_blocks) * FLOW_DEPS, 0);
    auto overlap = [len](long long s1, long long e1, long long s2, long long e2) {
        if (e1 - s1 >= len || e2 - s2 >= len) return true;
        for (long long k = -2; k <= 2; ++k)
            if (s1 + k * len < e2 && s2 < e1 + k * len) return true;
        return false;
    };
    auto ws = [&](int a) { return (long long)a * width; };
    auto we = [&](int a) { return std::min(len, (long long)a * width + width); };
    for (int a = 0; a < n_blocks; ++a) {
        int cand[7], nc = 0;
        if (n_blocks <= 7) {
            for (int b = 0; b < n_blocks; ++b) cand[nc++] = b;
        } else {
            for (int d = -3; d <= 3; ++d) cand[nc++] = ((a + d) % n_blocks + n_blocks) % n_blocks;
        }
        int cnt = 0;
        for (int t = 0; t < nc; ++t) {
            const int b = cand[t];
            if (!overlap(ws(a) - lo, read_end(a), ws(b), we(b)) &&
                !overlap(ws(b) - lo, read_end(b), ws(a), we(a)))
                continue;
            if (cnt == FLOW_DEPS - 1) return false;
            out[size_t(a) * FLOW_DEPS + 1 + cnt++] = b;
        }
        out[size_t(a) * FLOW_DEPS] = cnt;
    }
    return true;
}

}  // namespace march
}  // namespace qla
