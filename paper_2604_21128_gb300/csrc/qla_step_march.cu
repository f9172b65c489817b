// Marching QLA step kernel: one step of Eq. 2e14 per launch, state and
// coefficients in registers, input rows staged through shared memory.
//
// Each warp owns a window of 32*LX columns (LX consecutive columns per lane)
// and marches down a segment of rows.  The window overlaps its neighbours by
// 4 columns on each side: U_x reaches four cells along x (four of its eight
// collision layers pair neighbouring sites), so the outer 4 columns of each
// side are recomputed halo and only the inner 32*LX - 8 columns are stored.
//
// Row by row:
//  * U_x (Eq. 2e6) acts on the whole row in registers.  Its eight layers are
//    disjoint 2x2 rotations (see layer_of); a bond that crosses a lane
//    boundary is computed by the lane that owns the bond's site, after one
//    shuffle brings the partner value in and one sends the result back.
//  * U_y (Eq. 2e9) runs as a software pipeline along y.  A layer that pairs
//    site j with j-1 or j+1 can finish row r-1 only when row r arrives, so
//    each of the four neighbour layers delays its output by one row and
//    carries two values per pair and column.  The output row of U_y is four
//    rows behind the input row, with no y-halo to recompute.
//  * V_x, V_y (Eqs. 2e11-2e13) of a step are applied when its output row
//    next enters a launch (before U_x), so the stored buffer holds
//    U_y U_x Q and the sequence of operations on the data is that of Eq. 2e14;
//    read-outs apply the pending V (see qla_ctx::pending_v).  Planes that U_y
//    does not touch are stored right after U_x, the others four rows later.
// The collision coefficients of the four rows in flight sit in a register
// ring; records come from the medium table through a 4-byte index per site.
// Rows are staged three ahead into a per-warp shared-memory ring by per-lane
// cp.async copies (no registers held while the loads fly); the next row's
// records are looked up one iteration early.  The march loop is unrolled by
// four so that every ring slot is a fixed register or buffer.
#include <algorithm>
#include <map>
#include <vector>

#include "qla_march2.cuh"
#include "qla_plateau.cuh"

namespace qla {
namespace {

using namespace march;

// Blocks per SM the register allocation must allow: the two-column
// variants in FP32 (E_z and six planes) and in FP64 E_z are held to 128
// registers (16 warps per SM).  Measured at 8192^2 against what they take
// unconstrained (3 blocks): FP32 six planes 11% faster (149 registers, a few
// bytes of spills at 128), FP64 E_z 10% (164 registers, a few hundred bytes
// of spills; the extra warps hide the FP64 pipe's result latency).  FP64 six
// planes (246) and double-single keep what they need.
template <typename T, int P, int LX> constexpr int min_blocks() {
    return LX == 2 && (std::is_same<T, float>::value ||
                       (std::is_same<T, double>::value && P == 3))
               ? 4
               : 1;
}

template <typename T, int P, int LX, int VM, bool VIN>
__global__ void __launch_bounds__(32 * WARPS, min_blocks<T, P, LX>())
k_step_march(const T *__restrict__ in, T *__restrict__ out, const uint32_t *__restrict__ midx,
             const MedRec<T> *__restrict__ table, int nx, int ny, int pitch, size_t plane,
             int seg_h, int n_wx, int n_items) {
    using M = March<T, P, LX, VM, VIN>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename M::Slot *ring =
        reinterpret_cast<typename M::Slot *>(smem_raw) + (threadIdx.x >> 5) * NSLOT;
    M m;
    m.in = in;
    m.out = out;
    m.midx = midx;
    m.table = table;
    m.pitch = pitch;
    m.plane = uint32_t(plane);
    m.total = uint32_t(ny) * uint32_t(pitch);
    const int item = blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (item < n_items) m.run_item(nx, ny, seg_h, n_wx, item, ring);
}

// The packed-pair variant (FP32 E_z; see qla_march2.cuh): same arguments.
template <int VM, bool VIN, typename PO, int MINB = 4, bool ILV = false>
__global__ void __launch_bounds__(32 * WARPS, MINB)
k_step_march2(const float *__restrict__ in, float *__restrict__ out,
              const uint32_t *__restrict__ midx, const MedRec<float> *__restrict__ table,
              int nx, int ny, int pitch, size_t plane, int seg_h, int n_wx, int n_items) {
    using M = March2<VM, VIN, PO, ILV>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename M::Slot *ring =
        reinterpret_cast<typename M::Slot *>(smem_raw) + (threadIdx.x >> 5) * NSLOT;
    M m;
    m.in = in;
    m.out = out;
    m.midx = midx;
    m.table = table;
    m.pitch = pitch;
    m.plane = uint32_t(plane);
    m.total = uint32_t(ny) * uint32_t(pitch);
    const int item = blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (item < n_items) m.run_item(nx, ny, seg_h, n_wx, item, ring);
}

// The plateau-split step (FP32 E_z; see qla_plateau.cuh): warp w of block b
// runs units[4 b + w].  The other units come first in the list, so the
// slower two-column work starts early and the plateau units fill the tail.
template <int VM, bool VIN>
__global__ void __launch_bounds__(32 * WARPS, 4)
k_step_march_split(const float *__restrict__ in, float *__restrict__ out,
                   const uint32_t *__restrict__ midx, const MedRec<float> *__restrict__ table,
                   int nx, int ny, int pitch, size_t plane, const int4 *__restrict__ units,
                   int n_units) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    const int li = int(blockIdx.x) * WARPS + warp;
    if (li >= n_units) return;   // the whole warp: units are per warp
    run_plateau_unit<VM, VIN>(in, out, midx, table, nx, ny, pitch, uint32_t(plane), units[li],
                              smem_raw + warp * plateau_ring_bytes<VM, VIN>());
}

// Dataflow steps of the plateau split (see flow_wait): n_steps steps of
// the unit list in one persistent launch, buffers a (the input of even
// steps) and b.  Blocks take four consecutive units w .. w + 3 (w = s *
// n_units + k) from the counter ctr[0], one per warp: neighbouring windows
// of one segment then start together, as the blocks of a per-step launch
// do, and the sectors they share at their edges are read once from DRAM
// (warps taking units one by one started them apart in time and read 20%
// more).  Odd steps start half-way down the lattice (k + shift), so that
// the first units of a step depend on units handed out half a step earlier
// rather than on the last ones of the step before.  done = ctr + 4: one
// counter per item.  A warp whose wait ran out (or that finds *err raised)
// skips its unit but still counts it, so the launch drains.
template <int VM>
__global__ void __launch_bounds__(32 * WARPS, 4)
k_step_march_flow(float *a, float *b, const uint32_t *__restrict__ midx,
                  const MedRec<float> *__restrict__ table, int nx, int ny, int pitch,
                  size_t plane, const int4 *__restrict__ units, int n_units, int seg, int n_wx,
                  int shift, const int *__restrict__ xdep, const int *__restrict__ ydep,
                  unsigned *ctr, int *err, int n_steps, long long budget, long long withhold) {
    constexpr bool VIN = VM != V_NONE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned s_w;
    __shared__ int s_e;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *ring = smem_raw + warp * plateau_ring_bytes<VM, VIN>();
    unsigned *done = ctr + 4;
    const unsigned total = unsigned(n_units) * unsigned(n_steps);
    for (;;) {
        __syncthreads();   // every warp has read the previous group
        if (threadIdx.x == 0) {
            s_w = atomicAdd(ctr, unsigned(WARPS));
            s_e = *static_cast<volatile int *>(err);
        }
        __syncthreads();
        if (s_w >= total) break;   // the whole block
        const unsigned w = s_w + unsigned(warp);
        if (w >= total) continue;
        const int s = int(w / unsigned(n_units));
        int k = int(w - unsigned(s) * unsigned(n_units));
        if (s & 1) {
            k += shift;
            if (k >= n_units) k -= n_units;
        }
        const int4 u = units[k];
        const int wx = u.x / PWOUT, wy = u.z / seg;
        bool go = s_e == 0;
        if (go && s > 0)
            go = flow_wait(xdep, ydep, done, n_wx, wx, wy, 6u * unsigned(s), err, budget);
        if (go)
            run_plateau_unit<VM, VIN>((s & 1) ? b : a, (s & 1) ? a : b, midx, table, nx, ny,
                                      pitch, uint32_t(plane), u, ring);
        // publish: every lane's stores, then the item's counter
        __syncwarp();
        if (lane == 0 && (long long)w != withhold) {
            __threadfence();
            atomicAdd(done + (wy * n_wx + wx), flow_increment(u, nx, wx));
        }
    }
}

// The double-single plateau split (E_z): the same units at 64-column
// windows.  The record-ring march of the other units needs 194 registers;
// holding the kernel to 3 or 4 blocks per SM made those units spill and the
// step slower (8192^2 ellipse: 3.37 and 3.40 ms against 2.59 ms at 2 blocks
// and 2.69 ms unsplit).
template <int VM, bool VIN>
__global__ void __launch_bounds__(32 * WARPS, 2)
k_step_march_split_ds(const dsf *__restrict__ in, dsf *__restrict__ out,
                      const uint32_t *__restrict__ midx, const MedRec<dsf> *__restrict__ table,
                      int nx, int ny, int pitch, size_t plane, const int4 *__restrict__ units,
                      int n_units) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    const int li = int(blockIdx.x) * WARPS + warp;
    if (li >= n_units) return;
    constexpr size_t ring = sizeof(typename March<dsf, 3, 2, VM, VIN, false>::Slot) * NSLOT;
    run_ds_unit<VM, VIN>(in, out, midx, table, nx, ny, pitch, uint32_t(plane), units[li],
                         smem_raw + warp * ring);
}

// Segment height: about two work items per resident warp slot (measured
// on the 8192^2 lattice: one exact wave leaves the schedulers less slack
// than two), rows a multiple of 4 and at least 32.  Within 25% of that
// target the count of segments that leaves the least ragged last segment
// wins (8192 rows: 32 segments of 256 rather than 33 of 252, whose short
// last segment idles its warps; 2% faster measured).
inline int pick_segment(int ny, int n_wx, long long resident_warps, int min_seg = 32) {
    if (resident_warps < 1) resident_warps = 1;
    long long target = 2 * resident_warps / n_wx;
    // more segments than min_seg-row ones all give the same height (and the
    // search below runs once per step launch: small lattices with large
    // targets cost ~15 us of host time per step before this cap)
    target = std::min<long long>(target, (ny + min_seg - 1) / min_seg);
    if (target < 1) target = 1;
    auto seg_for = [&](long long n_wy) {
        int seg = int((ny + n_wy - 1) / n_wy);
        if (seg < min_seg) seg = min_seg;
        return (seg + 3) / 4 * 4;
    };
    int best = seg_for(target);
    long long best_waste = -1, best_dist = 0;
    for (long long n = target - target / 4; n <= target + target / 4; ++n) {
        if (n < 1) continue;
        const int seg = seg_for(n);
        const long long used = (ny + seg - 1) / seg;
        const long long waste = used * seg - ny;
        const long long dist = n > target ? n - target : target - n;
        if (best_waste < 0 || waste < best_waste || (waste == best_waste && dist < best_dist)) {
            best = seg;
            best_waste = waste;
            best_dist = dist;
        }
    }
    return best;
}

// Kernel, staged-row size and stored columns per window of a variant; LX = 1
// selects the packed-pair kernel (FP32 E_z).
template <typename T, int P, int LX, int VM, bool VIN> struct Variant {
    static constexpr int WOUT = 32 * LX - 8;
    static constexpr size_t SLOT = sizeof(typename March<T, P, LX, VM, VIN>::Slot);
    static constexpr auto kern = k_step_march<T, P, LX, VM, VIN>;
};
template <typename PO, int VM, bool VIN, int MINB = 4, bool ILV = false> struct Variant2 {
    static constexpr int WOUT = March2<VM, VIN, PO, ILV>::WOUT;
    static constexpr size_t SLOT = sizeof(typename March2<VM, VIN, PO, ILV>::Slot);
    static constexpr auto kern = k_step_march2<VM, VIN, PO, MINB, ILV>;
};
template <int VM, bool VIN> struct Variant<float, 3, 1, VM, VIN> : Variant2<PairF2, VM, VIN> {};
template <int VM, bool VIN> struct Variant<float, 3, 5, VM, VIN> : Variant2<PairF2, VM, VIN, 4, true> {};

// The plateau plan for segments of `seg` rows: classify the plateau-window
// items and write the unit list to c->items (the other items' units first,
// then the plateau units).  With `flow`, the units go in item order (rows of
// items top to bottom), followed by the dataflow tables; the plan is left
// unbuilt if they do not fit.  Synchronises the context's stream once.
cudaError_t build_plateau_plan(qla_ctx *c, int seg, bool flow) {
    auto &u = c->uplan;
    u.gen = -1;
    u.n_uniform = 0;
    u.flow = false;
    const int n_wx = (c->nx + PWOUT - 1) / PWOUT;
    const int n_wy = (c->ny + seg - 1) / seg;
    const int n_items = n_wx * n_wy;
    // capacity: three units per item at most
    if (size_t(3) * n_items > c->items_cap) return cudaSuccess;
    int *cls_dev = reinterpret_cast<int *>(c->items);
    k_classify_items<<<(n_items + WARPS - 1) / WARPS, 32 * WARPS, 0, c->stream>>>(
        c->midx, c->nx, c->ny, c->pitch, seg, n_wx, n_items, cls_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::vector<int> cls(n_items);
    e = cudaMemcpyAsync(cls.data(), cls_dev, size_t(n_items) * 4, cudaMemcpyDeviceToHost,
                        c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    std::vector<int4> list, plat;
    list.reserve(size_t(3) * n_items);
    int n_plateau = 0;
    if (flow) {
        // item order: each item's units together, rows of items in turn
        for (int i = 0; i < n_items; ++i) {
            const int wx = i % n_wx, wy = i / n_wx;
            const int x_out = wx * PWOUT, w_out = std::min(PWOUT, c->nx - x_out);
            const int y_lo = wy * seg, y_hi = std::min(c->ny, y_lo + seg);
            if (cls[i] >= 0) {
                list.push_back(plateau_unit(x_out, w_out, cls[i], y_lo, y_hi));
                ++n_plateau;
            } else {
                for (int x = x_out; x < x_out + w_out; x += GWOUT)
                    list.push_back(
                        plateau_unit(x, std::min(GWOUT, x_out + w_out - x), -1, y_lo, y_hi));
            }
        }
    } else {
        n_plateau = plateau_units(cls, c->nx, c->ny, seg, list, plat);
        list.insert(list.end(), plat.begin(), plat.end());
    }
    std::vector<int> recs;
    for (int v : cls)
        if (v >= 0) recs.push_back(v);
    std::sort(recs.begin(), recs.end());
    const int n_recs = int(std::unique(recs.begin(), recs.end()) - recs.begin());
    // the bytes uploaded: the unit list, then (flow) the two dependency
    // tables; the counters follow and are cleared by each launch
    std::vector<char> blob(list.size() * sizeof(int4));
    memcpy(blob.data(), list.data(), blob.size());
    size_t off_xdep = 0, off_ydep = 0, off_ctr = 0;
    if (flow) {
        std::vector<int> xd, yd;
        const bool ok_x = flow_axis_deps(c->nx, PWOUT, n_wx, 4, [&](int a) {
            const long long x = (long long)a * PWOUT;
            const int w = int(std::min<long long>(PWOUT, c->nx - x));
            const int last = (w - 1) / GWOUT * GWOUT;   // start of the last two-column unit
            return x + std::max(PW - 4, last + 64 - 4);
        }, xd);
        const bool ok_y = flow_axis_deps(c->ny, seg, n_wy, LAG, [&](int a) {
            return std::min<long long>(c->ny, (long long)(a + 1) * seg) + LAG;
        }, yd);
        off_xdep = (blob.size() + 15) / 16 * 16;
        off_ydep = off_xdep + (xd.size() * 4 + 15) / 16 * 16;
        off_ctr = off_ydep + (yd.size() * 4 + 15) / 16 * 16;
        const size_t end = off_ctr + 16 + size_t(n_items) * 4;
        // the wait flag sits in the last 16 bytes of the region
        if (!ok_x || !ok_y || end + 16 > c->items_cap * sizeof(int4)) return cudaSuccess;
        blob.resize(off_ctr, 0);
        memcpy(blob.data() + off_xdep, xd.data(), xd.size() * 4);
        memcpy(blob.data() + off_ydep, yd.data(), yd.size() * 4);
    }
    e = cudaMemcpyAsync(c->items, blob.data(), blob.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    if (flow) {
        u.flow = true;
        u.n_wx = n_wx;
        // odd steps start at the first unit of segment n_wy / 2
        int shift = 0;
        while (shift < int(list.size()) && list[shift].z < (n_wy / 2) * seg) ++shift;
        u.shift = shift == int(list.size()) ? 0 : shift;
        u.off_xdep = off_xdep;
        u.off_ydep = off_ydep;
        u.off_ctr = off_ctr;
    }
    u.gen = c->medium_gen;
    u.seg = seg;
    u.n_items = n_items;
    u.n_list = int(list.size());
    u.n_uniform = n_plateau;
    u.n_sets = n_recs;
    return cudaSuccess;
}

// The double-single plan: items of 64-column windows (56 stored columns),
// one unit each, the other items first.  Synchronises the stream once.
cudaError_t build_plateau_plan_ds(qla_ctx *c, int seg) {
    auto &u = c->uplan;
    u.gen = -1;
    u.n_uniform = 0;
    const int n_wx = (c->nx + GWOUT - 1) / GWOUT;
    const int n_items = n_wx * ((c->ny + seg - 1) / seg);
    if (size_t(n_items) > c->items_cap) return cudaSuccess;
    int *cls_dev = reinterpret_cast<int *>(c->items);
    k_classify<2><<<(n_items + WARPS - 1) / WARPS, 32 * WARPS, 0, c->stream>>>(
        c->midx, c->nx, c->ny, c->pitch, seg, n_wx, n_items, cls_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::vector<int> cls(n_items);
    e = cudaMemcpyAsync(cls.data(), cls_dev, size_t(n_items) * 4, cudaMemcpyDeviceToHost,
                        c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    std::vector<int4> list, plat;
    std::vector<int> recs;
    for (int i = 0; i < n_items; ++i) {
        const int wx = i % n_wx, wy = i / n_wx;
        const int x_out = wx * GWOUT, w_out = std::min(GWOUT, c->nx - x_out);
        const int y_lo = wy * seg, y_hi = std::min(c->ny, y_lo + seg);
        (cls[i] >= 0 ? plat : list).push_back(plateau_unit(x_out, w_out, cls[i], y_lo, y_hi));
        if (cls[i] >= 0) recs.push_back(cls[i]);
    }
    const int n_plateau = int(plat.size());
    list.insert(list.end(), plat.begin(), plat.end());
    std::sort(recs.begin(), recs.end());
    const int n_recs = int(std::unique(recs.begin(), recs.end()) - recs.begin());
    e = cudaMemcpyAsync(c->items, list.data(), list.size() * sizeof(int4), cudaMemcpyHostToDevice,
                        c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    u.gen = c->medium_gen;
    u.seg = seg;
    u.n_items = n_items;
    u.n_list = int(list.size());
    u.n_uniform = n_plateau;
    u.n_sets = n_recs;
    return cudaSuccess;
}

// The dataflow launches' wait flag: the last 16 bytes of the unit region,
// which no plan uses, so it survives plan rebuilds until the host reads it.
int *flow_flag(qla_ctx *c) {
    return reinterpret_cast<int *>(reinterpret_cast<char *>(c->items) + c->items_cap * 16 - 16);
}

// The plan of segments of `seg` rows (dataflow order and tables with
// `flow`), built unless it is the current one.  A dataflow plan that does
// not fit the workspace falls back to the per-step plan of the same
// segments (and is not retried until the medium or the tuning changes).
cudaError_t ensure_plateau_plan(qla_ctx *c, int seg, bool flow) {
    auto &u = c->uplan;
    if (u.gen == c->medium_gen && u.seg == seg && u.want_flow == flow) return cudaSuccess;
    cudaError_t e = build_plateau_plan(c, seg, flow);
    if (e == cudaSuccess && flow && u.gen != c->medium_gen) e = build_plateau_plan(c, seg, false);
    if (e == cudaSuccess) u.want_flow = flow;
    return e;
}

// Segment height of the dataflow plan of an FP32 E_z context, or 0 where its
// steps run one launch each.  Dataflow steps need about three items per
// resident warp slot: a unit's dependencies are then handed out about 1.5
// waves before it (half a step, see k_step_march_flow) and have finished.
// Taller segments recompute fewer halo rows but leave less of that slack:
// without a tuning, the tallest segment of 64 to 256 rows (multiples of 32)
// with at least 4.5 items per slot, else 64 rows with at least three
// (measured on the 16384^2 vacuum bubble, per step: 1.375 ms at 192 rows
// with 4.8 items per slot, 1.395 ms at 256 rows with 3.6, 1.401 ms at 128
// rows with 7.2, against 1.415 ms for launches per step; 8192^2 ellipse:
// 0.398 ms at 64 rows with 3.6, against 0.403 ms).
// QLA_KERNEL_MARCH_FLOW takes dataflow steps on any lattice the plateau
// split takes (32-row segments where none gives three items per slot).
int flow_segment(const qla_ctx *c) {
    if (c->prec != QLA_FP32 || c->P != 3 || march_lane_cols(c) != 2 || !c->items ||
        c->nx % 4 != 0 || c->nx < PW)
        return 0;
    const int k = c->step_kernel;
    if (k != QLA_KERNEL_AUTO && k != QLA_KERNEL_MARCH && k != QLA_KERNEL_MARCH_FLOW) return 0;
    const long long n_wx = (c->nx + PWOUT - 1) / PWOUT;
    const long long slots = 4LL * WARPS * c->num_sms;
    // items x 2 >= slots x twice the target
    auto items2 = [&](int seg) { return 2 * n_wx * ((c->ny + seg - 1) / seg); };
    if (c->march_seg > 0) {
        const int seg = std::max(16, (c->march_seg + 3) / 4 * 4);
        return k == QLA_KERNEL_MARCH_FLOW || items2(seg) >= 6 * slots ? seg : 0;
    }
    for (int seg = 256; seg >= 64; seg -= 32)
        if (items2(seg) >= 9 * slots) return seg;
    if (items2(64) >= 6 * slots) return 64;
    return k == QLA_KERNEL_MARCH_FLOW ? 32 : 0;
}

template <int VM>
cudaError_t launch_flow(qla_ctx *c, const void *in, void *out, long long n_steps) {
    auto kern = k_step_march_flow<VM>;
    constexpr bool VIN = VM != V_NONE;
    const size_t smem = plateau_ring_bytes<VM, VIN>() * WARPS;
    struct Occ { cudaError_t err; int per_sm; };
    static const Occ occ = [&] {
        Occ o{cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
              1};
        int b = 0;
        if (o.err == cudaSuccess)
            o.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 32 * WARPS, smem);
        o.per_sm = b > 0 ? b : 1;
        return o;
    }();
    if (occ.err != cudaSuccess) return occ.err;
    const auto &u = c->uplan;
    char *base = reinterpret_cast<char *>(c->items);
    unsigned *ctr = reinterpret_cast<unsigned *>(base + u.off_ctr);
    int *err = flow_flag(c);
    if (!c->flow_unchecked) {
        const cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), c->stream);
        if (e != cudaSuccess) return e;
    }
    // units x steps of one launch below 2^31, item counters below 2^32
    const long long per = std::max(1LL, std::min<long long>((1LL << 31) / u.n_list, 1LL << 26));
    float *a = static_cast<float *>(const_cast<void *>(in)), *b = static_cast<float *>(out);
    for (long long left = n_steps; left > 0;) {
        const long long k = std::min(per, left);
        cudaError_t e = cudaMemsetAsync(ctr, 0, 16 + size_t(u.n_items) * 4, c->stream);
        if (e != cudaSuccess) return e;
        kern<<<occ.per_sm * c->num_sms, 32 * WARPS, smem, c->stream>>>(
            a, b, c->midx, static_cast<const MedRec<float> *>(c->table), c->nx, c->ny, c->pitch,
            c->plane_elems, reinterpret_cast<const int4 *>(c->items), u.n_list, u.seg, u.n_wx,
            u.shift, reinterpret_cast<const int *>(base + u.off_xdep),
            reinterpret_cast<const int *>(base + u.off_ydep), ctr, err, int(k), c->flow_budget,
            c->flow_withhold);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        c->launches++;
        c->flow_unchecked = true;
        if (k & 1) std::swap(a, b);
        left -= k;
    }
    return cudaSuccess;
}

template <int VM, bool VIN>
cudaError_t launch_split_ds(qla_ctx *c, const void *in, void *out) {
    auto kern = k_step_march_split_ds<VM, VIN>;
    const size_t smem = sizeof(typename March<dsf, 3, 2, VM, VIN, false>::Slot) * NSLOT * WARPS;
    static const cudaError_t attr =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (attr != cudaSuccess) return attr;
    const auto &u = c->uplan;
    kern<<<(u.n_list + WARPS - 1) / WARPS, 32 * WARPS, smem, c->stream>>>(
        static_cast<const dsf *>(in), static_cast<dsf *>(out), c->midx,
        static_cast<const MedRec<dsf> *>(c->dstable), c->nx, c->ny, c->pitch, c->plane_elems,
        reinterpret_cast<const int4 *>(c->items), u.n_list);
    return cudaGetLastError();
}

template <int VM, bool VIN>
cudaError_t launch_split(qla_ctx *c, const void *in, void *out) {
    auto kern = k_step_march_split<VM, VIN>;
    const size_t smem = plateau_ring_bytes<VM, VIN>() * WARPS;
    static const cudaError_t attr =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (attr != cudaSuccess) return attr;
    const auto &u = c->uplan;
    kern<<<(u.n_list + WARPS - 1) / WARPS, 32 * WARPS, smem, c->stream>>>(
        static_cast<const float *>(in), static_cast<float *>(out), c->midx,
        static_cast<const MedRec<float> *>(c->table), c->nx, c->ny, c->pitch, c->plane_elems,
        reinterpret_cast<const int4 *>(c->items), u.n_list);
    return cudaGetLastError();
}

template <typename T, int P, int LX, int VM, bool VIN>
cudaError_t launch_t(qla_ctx *c, const void *in, void *out, const void *table) {
    using V = Variant<T, P, LX, VM, VIN>;
    constexpr int WOUT = V::WOUT;
    auto kern = V::kern;
    const size_t smem = V::SLOT * NSLOT * WARPS;
    // per instantiation, per process; initialised once (thread-safe)
    struct Occ { cudaError_t err; int per_sm; };
    static const Occ occ = [&] {
        Occ o{cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
              1};
        int b = 0;
        if (o.err == cudaSuccess)
            o.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 32 * WARPS, smem);
        o.per_sm = b > 0 ? b : 1;
        return o;
    }();
    if (occ.err != cudaSuccess) return occ.err;
    const int blocks_per_sm = occ.per_sm;
    const int n_wx = (c->nx + WOUT - 1) / WOUT;
    int seg = c->march_seg;
    if (seg <= 0) {
        long long resident = (long long)blocks_per_sm * WARPS * c->num_sms;
        // FP64 E_z is bound by the FP64 pipe, which few warps keep busy, while
        // every segment re-reads 8 rows: half an item per resident warp slot
        // measured best (8192^2: 1024-row segments 8.6e9 site-updates/s
        // against 8.4e9 at 256; 4096^2: 256 rows 8.4e9 against 7.7e9 at 64)
        if (std::is_same<T, double>::value && P == 3) resident /= 4;
        seg = pick_segment(c->ny, n_wx, resident);
    } else {
        seg = (seg + 3) / 4 * 4;
    }
    const int n_wy = (c->ny + seg - 1) / seg;
    const int n_items = n_wx * n_wy;
    if constexpr (std::is_same<T, float>::value && P == 3 && LX == 2) {
        if (c->items && c->step_kernel != QLA_KERNEL_MARCH_PLAIN && table == c->table &&
            c->nx % 4 == 0 && c->nx >= PW) {
            // plateau windows are 120 columns wide: segments for about eight
            // of them per resident warp slot, of at least 64 rows (measured
            // per step: 16384^2 vacuum bubble 1.51 ms at 96-128 rows, 1.54 at
            // 256, 1.65 at 512; 8192^2 ellipse 0.430 ms at 64 rows, 0.453 at
            // 128, 0.467 at 256)
            const int fseg = flow_segment(c);
            int pseg = fseg > 0 ? fseg : c->march_seg;
            if (pseg <= 0) {
                const int n_pwx = (c->nx + PWOUT - 1) / PWOUT;
                const long long slots = (long long)blocks_per_sm * WARPS * c->num_sms;
                // lattices with less than a wave of 64-row items (256^2: 12)
                // are latency-bound: shorter segments give more warps
                const int min_seg = (long long)((c->ny + 63) / 64) * n_pwx >= slots ? 64 : 16;
                pseg = pick_segment(c->ny, n_pwx, 4 * slots, min_seg);
            } else {
                pseg = (pseg + 3) / 4 * 4;
            }
            const auto &u = c->uplan;
            if (pseg >= 16) {
                const cudaError_t e = ensure_plateau_plan(c, pseg, fseg > 0);
                if (e != cudaSuccess) return e;
            }
            if (u.gen == c->medium_gen && u.seg == pseg && u.n_uniform > 0)
                return launch_split<VM, VIN>(c, in, out);
        }
    }
    if constexpr (std::is_same<T, dsf>::value && P == 3 && LX == 2) {
        if (c->items && c->step_kernel != QLA_KERNEL_MARCH_PLAIN && table == c->dstable) {
            // about four items per resident warp slot (2 blocks per SM): the
            // other items take longer than plateau items, and one wave of
            // mixed items leaves a tail (8192^2 ellipse: 2.59 ms per step at
            // 256-row segments, 3.46 ms at the unsplit kernel's 512)
            const int dseg = c->march_seg > 0
                                 ? seg
                                 : pick_segment(c->ny, n_wx, 4LL * WARPS * c->num_sms);
            const auto &u = c->uplan;
            if (dseg >= 16 && (u.gen != c->medium_gen || u.seg != dseg)) {
                const cudaError_t e = build_plateau_plan_ds(c, dseg);
                if (e != cudaSuccess) return e;
            }
            if (u.gen == c->medium_gen && u.seg == dseg && u.n_uniform > 0)
                return launch_split_ds<VM, VIN>(c, in, out);
        }
    }
    const int blocks = (n_items + WARPS - 1) / WARPS;
    kern<<<blocks, 32 * WARPS, smem, c->stream>>>(
        static_cast<const T *>(in), static_cast<T *>(out), c->midx,
        static_cast<const MedRec<T> *>(table), c->nx, c->ny, c->pitch, c->plane_elems, seg,
        n_wx, n_items);
    return cudaGetLastError();
}

// The previous step's potential operator is applied to each entering row
// when one is pending (see qla_ctx::pending_v).
template <typename T, int P, int LX>
cudaError_t launch_vm(qla_ctx *c, const void *in, void *out, bool vin) {
    const void *tb = c->table;
    switch (c->vmode) {
    case V_ROTATION:
        return vin ? launch_t<T, P, LX, V_ROTATION, true>(c, in, out, tb)
                   : launch_t<T, P, LX, V_ROTATION, false>(c, in, out, tb);
    case V_LITERAL:
        return vin ? launch_t<T, P, LX, V_LITERAL, true>(c, in, out, tb)
                   : launch_t<T, P, LX, V_LITERAL, false>(c, in, out, tb);
    default: return launch_t<T, P, LX, V_NONE, false>(c, in, out, tb);
    }
}

// Double-single steps: word-pair state, MedRec<dsf> records; the rotation
// or no-potential reading (the flag excludes the others).
template <int P>
cudaError_t launch_ds(qla_ctx *c, const void *in, void *out, bool vin) {
    const void *tb = c->dstable;
    if (c->vmode == V_ROTATION)
        return vin ? launch_t<dsf, P, 2, V_ROTATION, true>(c, in, out, tb)
                   : launch_t<dsf, P, 2, V_ROTATION, false>(c, in, out, tb);
    return launch_t<dsf, P, 2, V_NONE, false>(c, in, out, tb);
}

}  // namespace

// Column layout for FP32 E_z contexts: 1 = the packed-pair kernel (two
// columns 32 apart per lane, FP32x2 arithmetic), 5 = the same with U_x of
// the next row interleaved with U_y of the current one, or 2 or 4 adjacent
// columns per lane (scalar arithmetic; 2 is the default: at 128 registers
// four warps per scheduler stay resident, which outweighs the wider
// window's smaller halo, and the packed forms measured no faster).
// Other contexts: 2.
int march_lane_cols(const qla_ctx *c) {
    if (c->prec == QLA_FP32 && c->P == 3 && c->march_lx != 0) return c->march_lx;
    return 2;
}

bool march_supported(const qla_ctx *c) {
    const int lx = march_lane_cols(c);
    const bool packed = lx == 1 || lx == 5;
    const int align = packed ? 4 : lx, width = packed ? 64 : 32 * lx;
    return c->nx % align == 0 && c->nx >= width && c->ny >= 8 &&
           c->plane_elems < (size_t(1) << 31) && !(c->tensor && c->P == 6) &&
           c->vmode != V_LCU;
}

bool ds_shape_ok(int nx, int ny) {
    return nx % 2 == 0 && nx >= 64 && ny >= 8 &&
           size_t(ny) * ((size_t(nx) + 31) / 32 * 32) < (size_t(1) << 31);
}

// Six-plane double-single steps run as two launches, one per decoupled
// triple (P_TE6, then P_TM6), each with the E_z kernel's register budget:
// a single six-plane launch needs 255 registers (two blocks per SM) and
// reached a quarter of the E_z rate.  The arithmetic per pair is unchanged.
cudaError_t launch_step_march_ds(qla_ctx *c, const void *in, void *out, bool vin) {
    if (c->P != 6) return launch_ds<3>(c, in, out, vin);
    const cudaError_t e = launch_ds<P_TE6>(c, in, out, vin);
    return e != cudaSuccess ? e : launch_ds<P_TM6>(c, in, out, vin);
}

int step_march_ds_launches(const qla_ctx *c) { return c->P == 6 ? 2 : 1; }

cudaError_t launch_step_march(qla_ctx *c, const void *in, void *out, bool vin) {
    if (c->prec == QLA_FP64)
        return c->P == 6 ? launch_vm<double, 6, 2>(c, in, out, vin)
                         : launch_vm<double, 3, 2>(c, in, out, vin);
    if (c->P == 6) return launch_vm<float, 6, 2>(c, in, out, vin);
    switch (march_lane_cols(c)) {
    case 1: return launch_vm<float, 3, 1>(c, in, out, vin);
    case 5: return launch_vm<float, 3, 5>(c, in, out, vin);
    case 4: return launch_vm<float, 3, 4>(c, in, out, vin);
    default: return launch_vm<float, 3, 2>(c, in, out, vin);
    }
}

cudaError_t launch_step_flow(qla_ctx *c, long long n_steps, bool *done) {
    *done = false;
    const int seg = flow_segment(c);
    if (seg <= 0 || n_steps < 1) return cudaSuccess;
    cudaError_t e = ensure_plateau_plan(c, seg, true);
    if (e != cudaSuccess) return e;
    const auto &u = c->uplan;
    if (u.gen != c->medium_gen || u.seg != seg || !u.flow || u.n_uniform == 0) return cudaSuccess;
    *done = true;
    if (!c->pending_v && c->vmode != V_NONE) {
        // the first step has no potential step to apply on entry: one
        // per-step launch (the same plan), the rest with it pending
        e = launch_step_march(c, c->state[c->cur], c->state[c->cur ^ 1], false);
        if (e != cudaSuccess) return e;
        c->launches++;
        c->cur ^= 1;
        c->pending_v = true;
        if (--n_steps == 0) return cudaSuccess;
    }
    const void *in = c->state[c->cur];
    void *out = c->state[c->cur ^ 1];
    switch (c->vmode) {
    case V_ROTATION: e = launch_flow<V_ROTATION>(c, in, out, n_steps); break;
    case V_LITERAL: e = launch_flow<V_LITERAL>(c, in, out, n_steps); break;
    default: e = launch_flow<V_NONE>(c, in, out, n_steps); break;
    }
    if (e != cudaSuccess) return e;
    if (n_steps & 1) c->cur ^= 1;
    c->pending_v = c->vmode != V_NONE;
    return cudaSuccess;
}

cudaError_t flow_timed_out(qla_ctx *c, bool *timed_out) {
    *timed_out = false;
    if (!c->flow_unchecked) return cudaSuccess;
    int v = 0;
    const cudaError_t e = cudaMemcpy(&v, flow_flag(c), sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    c->flow_unchecked = false;
    *timed_out = v != 0;
    return cudaSuccess;
}

}  // namespace qla
