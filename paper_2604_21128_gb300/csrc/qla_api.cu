// C ABI of libqla (declared in include/qla.h): argument checking, the
// workspace layout, host <-> device copies and the step loop.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "qla_internal.h"
#include "qla_limits.h"
#include "qla_plateau.cuh"

namespace qla {

static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// The marching kernel takes the lattice and its 32-bit offsets reach every
// live plane.
static bool march_ok(const qla_ctx *c) {
    return march_supported(c) && offsets32_ok(size_t(c->P), c->plane_elems);
}

Layout layout_for(int nx, int ny, int prec, unsigned flags) {
    Layout L{};
    const size_t elt = prec == QLA_FP64 ? 8 : 4;
    const int P = (flags & QLA_TE_ONLY) ? 3 : 6;
    // rows padded to 32 elements: 128-byte aligned rows for FP32, 256 for FP64
    L.pitch = (nx + 31) / 32 * 32;
    L.plane_elems = size_t(ny) * L.pitch;
    const size_t plane_bytes = align256(L.plane_elems * elt);
    const size_t rec = prec == QLA_FP64 ? sizeof(MedRec<double>) : sizeof(MedRec<float>);
    // energy partials: one per block of 256 threads x 8 sites, capped
    const size_t sites = size_t(nx) * ny;
    size_t nb = (sites + 2047) / 2048;
    if (nb > 4096) nb = 4096;
    if (nb < 1) nb = 1;
    L.energy_blocks = int(nb);
    size_t off = 0;
    L.state[0] = off; off += align256(plane_bytes * P);
    L.state[1] = off; off += align256(plane_bytes * P);
    L.midx = off;     off += align256(L.plane_elems * 4);
    L.table = off;    off += align256((UNIFORM_SLOTS + sites) * rec);
    L.keys = off;     off += align256(UNIFORM_SLOTS * 8);
    L.counter = off;  off += align256(4);
    L.n = off;        off += align256(L.plane_elems * 8);
    L.staging = off;  off += align256(sites * 8);
    // partials: up to DIV_TERMS doubles per block (energy uses one)
    L.partials = off; off += align256(nb * 8 * DIV_TERMS);
    L.result = off;   off += align256(8 * DIV_TERMS);
    L.n_x = L.n_y = L.ttable = 0;
    if (flags & QLA_ANISOTROPIC) {
        L.n_x = off; off += align256(L.plane_elems * 8);
        L.n_y = off; off += align256(L.plane_elems * 8);
        if (P == 6) {
            const size_t trec = prec == QLA_FP64 ? sizeof(MedRecT<double>) : sizeof(MedRecT<float>);
            L.ttable = off; off += align256(L.plane_elems * trec);
        }
    }
    L.dstable = 0;
    if ((flags & QLA_DOUBLE_SINGLE) && prec == QLA_FP64) {
        L.dstable = off; off += align256((UNIFORM_SLOTS + sites) * sizeof(MedRec<dsf>));
    }
    // FP32 E_z: the plateau-split step's unit list (int4 entries): three
    // units per 120-column window and segment of at least 16 rows
    L.items = L.items_cap = 0;
    if (prec == QLA_FP32 && P == 3) {
        L.items_cap = 3 * size_t((nx + 119) / 120) * size_t((ny + 15) / 16);
        L.items = off; off += align256(L.items_cap * 16);
    } else if (prec == QLA_FP64 && P == 3 && (flags & QLA_DOUBLE_SINGLE)) {
        // double-single E_z: one unit per 56-column window and segment
        L.items_cap = size_t((nx + 55) / 56) * size_t((ny + 15) / 16);
        L.items = off; off += align256(L.items_cap * 16);
    }
    L.total = off;
    return L;
}

}  // namespace qla

using namespace qla;

namespace {

qla_status fail(qla_ctx *c, qla_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
qla_status fail(qla_ctx *c, qla_status s, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
        if (s == QLA_ECUDA) c->sticky = QLA_ECUDA;
    }
    return s;
}

qla_status cuda_fail(qla_ctx *c, cudaError_t e, const char *what) {
    return fail(c, QLA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define QLA_CUDA(c, call, what)                              \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, (what)); \
    } while (0)

// Make the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

// After a synchronisation of the context's stream: QLA_ETIMEOUT if a
// dataflow step launched since the last check gave up a dependency wait.
qla_status check_flow(qla_ctx *c, const char *what) {
    bool t = false;
    const cudaError_t e = flow_timed_out(c, &t);
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    if (t)
        return fail(c, QLA_ETIMEOUT,
                    "%s: a dataflow step's dependency wait ran out; the state is undefined "
                    "until it is set again", what);
    return QLA_OK;
}

qla_status usable(qla_ctx *c) {
    if (!c) return QLA_EINVAL;
    if (c->sticky != QLA_OK) return c->sticky;
    return QLA_OK;
}

}  // namespace

extern "C" {

size_t qla_workspace_bytes(int nx, int ny, int precision, unsigned flags) {
    if (nx < 1 || ny < 1 || (precision != QLA_FP64 && precision != QLA_FP32)) return 0;
    if (!record_ids_ok(size_t(nx) * size_t(ny), UNIFORM_SLOTS)) return 0;
    if ((flags & QLA_DOUBLE_SINGLE) &&
        (precision != QLA_FP64 ||
         (flags & (QLA_ANISOTROPIC | QLA_POTENTIAL_LITERAL | QLA_POTENTIAL_LCU)) ||
         !ds_shape_ok(nx, ny) ||
         !offsets32_ok((flags & QLA_TE_ONLY) ? 3 : 6, padded_plane(nx, ny))))
        return 0;
    return layout_for(nx, ny, precision, flags).total;
}

qla_status qla_init_grid(qla_ctx **out, int nx, int ny, double delta, int precision,
                         unsigned flags, void *cuda_stream, void *workspace,
                         size_t workspace_bytes) {
    if (!out) return QLA_EINVAL;
    *out = nullptr;
    if (nx < 1 || ny < 1 || !(delta > 0.0) || !std::isfinite(delta)) return QLA_EINVAL;
    if (precision != QLA_FP64 && precision != QLA_FP32) return QLA_EINVAL;
    if (flags & ~(unsigned)(QLA_TE_ONLY | QLA_POTENTIAL_LITERAL | QLA_POTENTIAL_NONE |
                            QLA_ANISOTROPIC | QLA_POTENTIAL_LCU | QLA_DOUBLE_SINGLE))
        return QLA_EINVAL;
    {
        const unsigned v = flags & (QLA_POTENTIAL_LITERAL | QLA_POTENTIAL_NONE | QLA_POTENTIAL_LCU);
        if (v & (v - 1)) return QLA_EINVAL;  // at most one potential reading
    }
    if ((flags & QLA_DOUBLE_SINGLE) &&
        (precision != QLA_FP64 || (flags & (QLA_ANISOTROPIC | QLA_POTENTIAL_LITERAL |
                                            QLA_POTENTIAL_LCU)) ||
         !ds_shape_ok(nx, ny) ||
         !offsets32_ok((flags & QLA_TE_ONLY) ? 3 : 6, padded_plane(nx, ny))))
        return QLA_EINVAL;
    if (!record_ids_ok(size_t(nx) * size_t(ny), UNIFORM_SLOTS)) return QLA_EINVAL;
    if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255)) return QLA_EINVAL;

    qla_ctx *c = new (std::nothrow) qla_ctx();
    if (!c) return QLA_ENOMEM;
    c->nx = nx;
    c->ny = ny;
    c->delta = delta;
    c->prec = precision;
    c->flags = flags;
    c->P = (flags & QLA_TE_ONLY) ? 3 : 6;
    c->vmode = (flags & QLA_POTENTIAL_LITERAL) ? V_LITERAL
             : (flags & QLA_POTENTIAL_NONE)    ? V_NONE
             : (flags & QLA_POTENTIAL_LCU)     ? V_LCU
                                               : V_ROTATION;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return QLA_ECUDA; }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);

    const Layout L = layout_for(nx, ny, precision, flags);
    if (workspace) {
        if (workspace_bytes < L.total) { delete c; return QLA_ENOMEM; }
        c->ws = static_cast<char *>(workspace);
        c->ws_bytes = workspace_bytes;
    } else {
        void *p = nullptr;
        if (cudaMalloc(&p, L.total) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return QLA_ENOMEM;
        }
        c->ws = static_cast<char *>(p);
        c->ws_bytes = L.total;
        c->owns_ws = true;
    }
    c->pitch = L.pitch;
    c->plane_elems = L.plane_elems;
    c->state[0] = c->ws + L.state[0];
    c->state[1] = c->ws + L.state[1];
    c->midx = reinterpret_cast<uint32_t *>(c->ws + L.midx);
    c->table = c->ws + L.table;
    c->keys = reinterpret_cast<unsigned long long *>(c->ws + L.keys);
    c->counter = reinterpret_cast<unsigned *>(c->ws + L.counter);
    c->n = reinterpret_cast<double *>(c->ws + L.n);
    c->staging = reinterpret_cast<double *>(c->ws + L.staging);
    c->partials = reinterpret_cast<double *>(c->ws + L.partials);
    c->result = reinterpret_cast<double *>(c->ws + L.result);
    c->energy_blocks = L.energy_blocks;
    c->tensor = (flags & QLA_ANISOTROPIC) != 0;
    if (c->tensor) {
        c->n_x = reinterpret_cast<double *>(c->ws + L.n_x);
        c->n_y = reinterpret_cast<double *>(c->ws + L.n_y);
        if (c->P == 6) c->ttable = c->ws + L.ttable;
    }
    if (flags & QLA_DOUBLE_SINGLE) c->dstable = c->ws + L.dstable;
    if (L.items_cap) {
        c->items = reinterpret_cast<int *>(c->ws + L.items);
        c->items_cap = L.items_cap;
    }
    // both state buffers start at zero (pad columns included)
    if (cudaMemsetAsync(c->ws + L.state[0], 0, L.midx - L.state[0], c->stream) != cudaSuccess) {
        cudaGetLastError();
        if (c->owns_ws) cudaFree(c->ws);
        delete c;
        return QLA_ECUDA;
    }
    *out = c;
    return QLA_OK;
}

static qla_status check_positive(qla_ctx *c, const double *a, const char *what) {
    const size_t N = size_t(c->nx) * c->ny;
    for (size_t k = 0; k < N; ++k) {
        const double v = a[k];
        if (!(v > 0.0) || !std::isfinite(v))
            return fail(c, QLA_EINVAL, "%s[%zu] = %g is not finite and > 0", what, k, v);
    }
    return QLA_OK;
}

qla_status qla_set_medium_tensor(qla_ctx *c, const double *n_x, const double *n_y,
                                 const double *n_z) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (!c->tensor)
        return fail(c, QLA_EINVAL, "qla_set_medium_tensor: context made without QLA_ANISOTROPIC");
    if (!n_x || !n_y || !n_z) return fail(c, QLA_EINVAL, "qla_set_medium_tensor: null array");
    if ((s = check_positive(c, n_x, "qla_set_medium_tensor: n_x")) != QLA_OK) return s;
    if ((s = check_positive(c, n_y, "qla_set_medium_tensor: n_y")) != QLA_OK) return s;
    if ((s = check_positive(c, n_z, "qla_set_medium_tensor: n_z")) != QLA_OK) return s;
    const size_t N = size_t(c->nx) * c->ny;
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_set_medium_tensor: cannot select device");
    // n_x and n_y through the staging plane into their pitched planes
    const double *src[2] = {n_x, n_y};
    double *dst[2] = {c->n_x, c->n_y};
    for (int k = 0; k < 2; ++k) {
        QLA_CUDA(c, cudaMemcpyAsync(c->staging, src[k], N * 8, cudaMemcpyHostToDevice, c->stream),
                 "qla_set_medium_tensor: copy");
        QLA_CUDA(c, launch_pitch_copy(c, dst[k]), "qla_set_medium_tensor: place");
    }
    // n_z is the scalar medium of the E_z triple: the shared-record table
    QLA_CUDA(c, cudaMemcpyAsync(c->staging, n_z, N * 8, cudaMemcpyHostToDevice, c->stream),
             "qla_set_medium_tensor: copy");
    QLA_CUDA(c, cudaMemsetAsync(c->keys, 0, UNIFORM_SLOTS * 8, c->stream),
             "qla_set_medium_tensor: clear");
    QLA_CUDA(c, cudaMemsetAsync(c->counter, 0, 4, c->stream), "qla_set_medium_tensor: clear");
    QLA_CUDA(c, launch_medium(c), "qla_set_medium_tensor: kernel");
    c->medium_gen++;
    if (c->P == 6) QLA_CUDA(c, launch_medium_tensor(c), "qla_set_medium_tensor: records");
    QLA_CUDA(c, cudaStreamSynchronize(c->stream), "qla_set_medium_tensor: sync");
    c->has_medium = true;
    return QLA_OK;
}

qla_status qla_set_medium(qla_ctx *c, const double *n_host) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (!n_host) return fail(c, QLA_EINVAL, "qla_set_medium: null n");
    if (c->tensor) return qla_set_medium_tensor(c, n_host, n_host, n_host);
    const size_t N = size_t(c->nx) * c->ny;
    for (size_t k = 0; k < N; ++k) {
        const double v = n_host[k];
        if (!(v > 0.0) || !std::isfinite(v))
            return fail(c, QLA_EINVAL, "qla_set_medium: n[%zu] = %g is not finite and > 0", k, v);
    }
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_set_medium: cannot select device");
    QLA_CUDA(c, cudaMemcpyAsync(c->staging, n_host, N * 8, cudaMemcpyHostToDevice, c->stream),
             "qla_set_medium: copy");
    QLA_CUDA(c, cudaMemsetAsync(c->keys, 0, UNIFORM_SLOTS * 8, c->stream), "qla_set_medium: clear");
    QLA_CUDA(c, cudaMemsetAsync(c->counter, 0, 4, c->stream), "qla_set_medium: clear");
    QLA_CUDA(c, launch_medium(c), "qla_set_medium: kernel");
    c->medium_gen++;
    c->has_medium = true;
    return QLA_OK;
}

qla_status qla_set_packet(qla_ctx *c, const qla_packet *p) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (!p) return fail(c, QLA_EINVAL, "qla_set_packet: null packet");
    const double v[7] = {p->x0, p->y0, p->angle, p->k0, p->width, p->transverse_width,
                         p->amplitude};
    for (double x : v)
        if (!std::isfinite(x)) return fail(c, QLA_EINVAL, "qla_set_packet: non-finite field");
    if (!(p->width > 0.0) || p->transverse_width < 0.0)
        return fail(c, QLA_EINVAL, "qla_set_packet: width must be > 0, transverse_width >= 0");
    if (!c->has_medium) return fail(c, QLA_ESTATE, "qla_set_packet: set the medium first");
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_set_packet: cannot select device");
    if (c->P == 6)
        QLA_CUDA(c, cudaMemsetAsync(c->state[c->cur], 0,
                                    c->plane_elems * (c->prec == QLA_FP64 ? 8 : 4) * 6, c->stream),
                 "qla_set_packet: clear");
    QLA_CUDA(c, launch_packet(c, *p), "qla_set_packet: kernel");
    c->has_state = true;
    c->pending_v = false;
    c->flow_unchecked = false;
    return QLA_OK;
}

qla_status qla_set_packet_window(qla_ctx *c, const qla_packet *p, int i0, int j0, int gnx,
                                 int gny) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (!p) return fail(c, QLA_EINVAL, "qla_set_packet_window: null packet");
    const double v[7] = {p->x0, p->y0, p->angle, p->k0, p->width, p->transverse_width,
                         p->amplitude};
    for (double x : v)
        if (!std::isfinite(x))
            return fail(c, QLA_EINVAL, "qla_set_packet_window: non-finite field");
    if (!(p->width > 0.0) || p->transverse_width < 0.0)
        return fail(c, QLA_EINVAL,
                    "qla_set_packet_window: width must be > 0, transverse_width >= 0");
    if (gnx < 1 || gny < 1 || i0 < 0 || j0 < 0 || i0 >= gnx || j0 >= gny)
        return fail(c, QLA_EINVAL, "qla_set_packet_window: window (%d, %d) of %d x %d", i0, j0,
                    gnx, gny);
    if (!c->has_medium) return fail(c, QLA_ESTATE, "qla_set_packet_window: set the medium first");
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_set_packet_window: cannot select device");
    if (c->P == 6)
        QLA_CUDA(c, cudaMemsetAsync(c->state[c->cur], 0,
                                    c->plane_elems * (c->prec == QLA_FP64 ? 8 : 4) * 6, c->stream),
                 "qla_set_packet_window: clear");
    QLA_CUDA(c, launch_packet_window(c, *p, i0, j0, gnx, gny), "qla_set_packet_window: kernel");
    c->has_state = true;
    c->pending_v = false;
    c->flow_unchecked = false;
    return QLA_OK;
}

size_t qla_box_bytes(const qla_ctx *c, int w, int h) {
    if (!c || w < 1 || h < 1 || w > c->nx || h > c->ny) return 0;
    return size_t(w) * size_t(h) * size_t(c->P) * (c->prec == QLA_FP64 ? 8 : 4);
}

}  // extern "C"

namespace {
qla_status box_args(qla_ctx *c, const char *who, int i0, int j0, int w, int h, const void *buf) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (!buf) return fail(c, QLA_EINVAL, "%s: null buffer", who);
    if (w < 1 || h < 1 || i0 < 0 || j0 < 0 || i0 > c->nx - w || j0 > c->ny - h)
        return fail(c, QLA_EINVAL, "%s: box (%d, %d) + %d x %d outside the %d x %d lattice", who,
                    i0, j0, w, h, c->nx, c->ny);
    if (!c->has_state) return fail(c, QLA_ESTATE, "%s: no state", who);
    return QLA_OK;
}
}  // namespace

extern "C" {

qla_status qla_pack_box(qla_ctx *c, int i0, int j0, int w, int h, void *dst_dev) {
    qla_status s = box_args(c, "qla_pack_box", i0, j0, w, h, dst_dev);
    if (s != QLA_OK) return s;
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_pack_box: cannot select device");
    QLA_CUDA(c, launch_box_copy(c, i0, j0, w, h, dst_dev, true), "qla_pack_box: kernel");
    return QLA_OK;
}

qla_status qla_unpack_box(qla_ctx *c, int i0, int j0, int w, int h, const void *src_dev) {
    qla_status s = box_args(c, "qla_unpack_box", i0, j0, w, h, src_dev);
    if (s != QLA_OK) return s;
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_unpack_box: cannot select device");
    QLA_CUDA(c, launch_box_copy(c, i0, j0, w, h, const_cast<void *>(src_dev), false),
             "qla_unpack_box: kernel");
    return QLA_OK;
}

qla_status qla_energy_box(qla_ctx *c, int i0, int j0, int w, int h, double *out) {
    qla_status s = box_args(c, "qla_energy_box", i0, j0, w, h, out);
    if (s != QLA_OK) return s;
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_energy_box: cannot select device");
    QLA_CUDA(c, launch_energy_box(c, i0, j0, w, h), "qla_energy_box: kernel");
    QLA_CUDA(c, cudaMemcpyAsync(out, c->result, 8, cudaMemcpyDeviceToHost, c->stream),
             "qla_energy_box: copy");
    QLA_CUDA(c, cudaStreamSynchronize(c->stream), "qla_energy_box: sync");
    {
        const qla_status f = check_flow(c, "qla_energy_box");
        if (f != QLA_OK) return f;
    }
    if (!std::isfinite(*out)) return fail(c, QLA_ENONFINITE, "qla_energy_box: energy is %g", *out);
    return QLA_OK;
}

qla_status qla_set_state(qla_ctx *c, const double *q_host) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (!q_host) return fail(c, QLA_EINVAL, "qla_set_state: null state");
    const size_t N = size_t(c->nx) * c->ny;
    for (size_t k = 0; k < 6 * N; ++k)
        if (!std::isfinite(q_host[k]))
            return fail(c, QLA_EINVAL, "qla_set_state: non-finite value at %zu", k);
    if (c->P == 3) {
        const int absent[3] = {0, 1, 5};
        for (int a : absent)
            for (size_t k = 0; k < N; ++k)
                if (q_host[size_t(a) * N + k] != 0.0)
                    return fail(c, QLA_EINVAL,
                                "qla_set_state: E_z context needs q%d == 0 (site %zu)", a, k);
    }
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_set_state: cannot select device");
    for (int comp = 0; comp < 6; ++comp) {
        const int plane = c->P == 6 ? comp : plane_of<3>(comp);
        if (plane < 0) continue;
        QLA_CUDA(c, cudaMemcpyAsync(c->staging, q_host + size_t(comp) * N, N * 8,
                                    cudaMemcpyHostToDevice, c->stream),
                 "qla_set_state: copy");
        QLA_CUDA(c, launch_from_f64(c, plane, c->staging), "qla_set_state: convert");
    }
    // the staging plane is reused per component: wait before the host buffer
    // may change and before the next copy overwrites staging
    QLA_CUDA(c, cudaStreamSynchronize(c->stream), "qla_set_state: sync");
    c->has_state = true;
    c->pending_v = false;
    c->flow_unchecked = false;   // a wait that ran out concerned the old state
    return QLA_OK;
}

qla_status qla_get_state(qla_ctx *c, double *q_host) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (!q_host) return fail(c, QLA_EINVAL, "qla_get_state: null output");
    const size_t N = size_t(c->nx) * c->ny;
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_get_state: cannot select device");
    for (int comp = 0; comp < 6; ++comp) {
        const int plane = c->P == 6 ? comp : plane_of<3>(comp);
        if (plane < 0) {
            std::memset(q_host + size_t(comp) * N, 0, N * 8);
            continue;
        }
        QLA_CUDA(c, launch_to_f64(c, comp, c->staging), "qla_get_state: convert");
        QLA_CUDA(c, cudaMemcpyAsync(q_host + size_t(comp) * N, c->staging, N * 8,
                                    cudaMemcpyDeviceToHost, c->stream),
                 "qla_get_state: copy");
        QLA_CUDA(c, cudaStreamSynchronize(c->stream), "qla_get_state: sync");
    }
    return check_flow(c, "qla_get_state");
}

qla_status qla_step(qla_ctx *c, long long n_steps) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (n_steps < 0) return fail(c, QLA_EINVAL, "qla_step: n_steps < 0");
    if (n_steps == 0) return QLA_OK;
    if (!c->has_medium || !c->has_state)
        return fail(c, QLA_ESTATE, "qla_step: set a medium and a state first");
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_step: cannot select device");
    if ((c->tensor && c->P == 6) || c->vmode == V_LCU) {
        // the tile kernel with this step's V applied in the same launch:
        // every pair with its own angle, or the LCU branches
        for (long long k = 0; k < n_steps; ++k) {
            QLA_CUDA(c, c->tensor && c->P == 6
                            ? launch_step_tensor(c, c->state[c->cur], c->state[c->cur ^ 1])
                            : launch_step_tile(c, c->state[c->cur], c->state[c->cur ^ 1], false),
                     "qla_step: kernel");
            c->launches++;
            c->cur ^= 1;
        }
        c->pending_v = false;
        return QLA_OK;
    }
    if (c->dstable) {
        // word pairs in place, n double-single steps, back to FP64
        QLA_CUDA(c, launch_state_to_ds(c, c->state[c->cur]), "qla_step: to double-single");
        c->launches++;
        for (long long k = 0; k < n_steps; ++k) {
            QLA_CUDA(c, launch_step_march_ds(c, c->state[c->cur], c->state[c->cur ^ 1],
                                             c->pending_v),
                     "qla_step: kernel");
            c->launches += step_march_ds_launches(c);
            c->cur ^= 1;
            c->pending_v = c->vmode != V_NONE;
        }
        QLA_CUDA(c, launch_state_from_ds(c, c->state[c->cur]), "qla_step: from double-single");
        c->launches++;
        return QLA_OK;
    }
    const bool march = c->step_kernel == QLA_KERNEL_MARCH ||
                       c->step_kernel == QLA_KERNEL_MARCH_PLAIN ||
                       c->step_kernel == QLA_KERNEL_MARCH_STEP ||
                       c->step_kernel == QLA_KERNEL_MARCH_FLOW ||
                       (c->step_kernel == QLA_KERNEL_AUTO && march_ok(c));
    if (march) {
        // all n steps in persistent dataflow launches where the context
        // takes them
        bool done = false;
        QLA_CUDA(c, launch_step_flow(c, n_steps, &done), "qla_step: dataflow kernel");
        if (done) return QLA_OK;
    }
    for (long long k = 0; k < n_steps; ++k) {
        const bool vin = c->pending_v;
        QLA_CUDA(c, march ? launch_step_march(c, c->state[c->cur], c->state[c->cur ^ 1], vin)
                          : launch_step_tile(c, c->state[c->cur], c->state[c->cur ^ 1], vin),
                 "qla_step: kernel");
        c->launches++;
        c->cur ^= 1;
        c->pending_v = c->vmode != V_NONE;
    }
    return QLA_OK;
}

qla_status qla_energy(qla_ctx *c, double *out) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (!out) return fail(c, QLA_EINVAL, "qla_energy: null output");
    if (!c->has_state) return fail(c, QLA_ESTATE, "qla_energy: no state");
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_energy: cannot select device");
    QLA_CUDA(c, launch_energy(c), "qla_energy: kernel");
    QLA_CUDA(c, cudaMemcpyAsync(out, c->result, 8, cudaMemcpyDeviceToHost, c->stream),
             "qla_energy: copy");
    QLA_CUDA(c, cudaStreamSynchronize(c->stream), "qla_energy: sync");
    {
        const qla_status f = check_flow(c, "qla_energy");
        if (f != QLA_OK) return f;
    }
    if (!std::isfinite(*out)) return fail(c, QLA_ENONFINITE, "qla_energy: energy is %g", *out);
    return QLA_OK;
}

qla_status qla_divergence(qla_ctx *c, double *out) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (!out) return fail(c, QLA_EINVAL, "qla_divergence: null output");
    if (!c->has_state || !c->has_medium)
        return fail(c, QLA_ESTATE, "qla_divergence: needs medium and state");
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_divergence: cannot select device");
    QLA_CUDA(c, launch_divergence(c), "qla_divergence: kernel");
    QLA_CUDA(c, cudaMemcpyAsync(out, c->result, 8 * DIV_TERMS, cudaMemcpyDeviceToHost, c->stream),
             "qla_divergence: copy");
    QLA_CUDA(c, cudaStreamSynchronize(c->stream), "qla_divergence: sync");
    {
        const qla_status f = check_flow(c, "qla_divergence");
        if (f != QLA_OK) return f;
    }
    for (int k = 0; k < DIV_TERMS; ++k)
        if (!std::isfinite(out[k]))
            return fail(c, QLA_ENONFINITE, "qla_divergence: term %d is %g", k, out[k]);
    return QLA_OK;
}

qla_status qla_fields(qla_ctx *c, double *Ex, double *Ey, double *Ez, double *Bx, double *By,
                      double *Bz) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (!c->has_state || !c->has_medium) return fail(c, QLA_ESTATE, "qla_fields: no state");
    double *outs[6] = {Ex, Ey, Ez, Bx, By, Bz};
    const size_t N = size_t(c->nx) * c->ny;
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_fields: cannot select device");
    for (int comp = 0; comp < 6; ++comp) {
        if (!outs[comp]) continue;
        QLA_CUDA(c, launch_fields(c, comp, c->staging), "qla_fields: kernel");
        QLA_CUDA(c, cudaMemcpyAsync(outs[comp], c->staging, N * 8, cudaMemcpyDeviceToHost,
                                    c->stream),
                 "qla_fields: copy");
        QLA_CUDA(c, cudaStreamSynchronize(c->stream), "qla_fields: sync");
    }
    return check_flow(c, "qla_fields");
}

qla_status qla_probe(qla_ctx *c, int count, const int *i, const int *j, double *out) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (count < 0 || count > 65536) return fail(c, QLA_EINVAL, "qla_probe: count %d", count);
    if (count == 0) return QLA_OK;
    if (!i || !j || !out) return fail(c, QLA_EINVAL, "qla_probe: null pointer");
    if (!c->has_state) return fail(c, QLA_ESTATE, "qla_probe: no state");
    std::vector<int> ij(2 * size_t(count));
    for (int k = 0; k < count; ++k) {
        if (i[k] < 0 || i[k] >= c->nx || j[k] < 0 || j[k] >= c->ny)
            return fail(c, QLA_EINVAL, "qla_probe: site %d = (%d, %d) outside the lattice", k,
                        i[k], j[k]);
        ij[k] = i[k];
        ij[count + k] = j[k];
    }
    // the staging plane (nx*ny doubles) holds the indices and the output;
    // a probe list larger than it is rejected
    const size_t need = 2 * size_t(count) * sizeof(int) + 6 * size_t(count) * sizeof(double) + 64;
    if (need > size_t(c->nx) * c->ny * 8)
        return fail(c, QLA_EINVAL, "qla_probe: %d sites do not fit this lattice's staging", count);
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, QLA_ECUDA, "qla_probe: cannot select device");
    double *dout = c->staging;
    int *dij = reinterpret_cast<int *>(c->staging + 6 * size_t(count));
    QLA_CUDA(c, cudaMemcpyAsync(dij, ij.data(), ij.size() * sizeof(int), cudaMemcpyHostToDevice,
                                c->stream),
             "qla_probe: copy in");
    QLA_CUDA(c, launch_probe(c, count, dij, dout), "qla_probe: kernel");
    QLA_CUDA(c, cudaMemcpyAsync(out, dout, 6 * size_t(count) * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream),
             "qla_probe: copy out");
    QLA_CUDA(c, cudaStreamSynchronize(c->stream), "qla_probe: sync");
    {
        const qla_status f = check_flow(c, "qla_probe");
        if (f != QLA_OK) return f;
    }
    return QLA_OK;
}

qla_status qla_set_step_kernel(qla_ctx *c, int kernel) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (kernel < QLA_KERNEL_AUTO || kernel > QLA_KERNEL_MARCH_FLOW)
        return fail(c, QLA_EINVAL, "qla_set_step_kernel: unknown kernel %d", kernel);
    const bool march = kernel != QLA_KERNEL_AUTO && kernel != QLA_KERNEL_TILE;
    if (march && ((c->tensor && c->P == 6) || c->vmode == V_LCU))
        return fail(c, QLA_EINVAL, "qla_set_step_kernel: six-plane tensor media and the LCU "
                                   "potential use the tile kernel");
    if (march && !march_ok(c))
        return fail(c, QLA_EINVAL, "qla_set_step_kernel: the marching kernel needs nx a multiple "
                                   "of its lane width (4 for the packed-pair layout), a window "
                                   "of columns and ny >= 8");
    c->step_kernel = kernel;
    return QLA_OK;
}

qla_status qla_set_march_tuning(qla_ctx *c, int lane_cols, int rows) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (lane_cols != 0 && lane_cols != 1 && lane_cols != 2 && lane_cols != 4 && lane_cols != 5)
        return fail(c, QLA_EINVAL, "qla_set_march_tuning: lane_cols %d not 0, 1, 2, 4 or 5",
                    lane_cols);
    if (rows < 0 || rows > (1 << 20))
        return fail(c, QLA_EINVAL, "qla_set_march_tuning: rows %d", rows);
    c->march_lx = lane_cols;
    c->march_seg = rows;
    return QLA_OK;
}

long long qla_launch_count(const qla_ctx *c) { return c ? c->launches : 0; }

qla_status qla_flow_plan(const qla_ctx *c, int *segment_rows) {
    if (!c || !segment_rows) return QLA_EINVAL;
    const auto &u = c->uplan;
    *segment_rows = u.gen == c->medium_gen && u.flow && u.n_uniform > 0 ? u.seg : 0;
    return QLA_OK;
}

qla_status qla_flow_item_deps(int nx, int ny, int segment_rows, int item, int *deps,
                              int capacity, int *count) {
    using namespace qla::march;
    if (!count || capacity < 0 || (capacity > 0 && !deps)) return QLA_EINVAL;
    *count = 0;
    if (nx < PW || nx % 4 != 0 || ny < 8 || segment_rows < 16 || segment_rows % 4 != 0)
        return QLA_EINVAL;
    const int seg = segment_rows;
    const int n_wx = (nx + PWOUT - 1) / PWOUT, n_wy = (ny + seg - 1) / seg;
    if (item < 0 || (long long)item >= (long long)n_wx * n_wy) return QLA_EINVAL;
    // the reads of the plan's items, as the dataflow plan takes them: a
    // window's 128 plateau columns from 4 left of its first stored column,
    // or its last two-column unit's 64 (from 4 left of that unit's first
    // stored column), whichever reaches further; a segment's rows and four
    // either side
    std::vector<int> xd, yd;
    const bool ok_x = flow_axis_deps(nx, PWOUT, n_wx, 4, [&](int a) {
        const long long x = (long long)a * PWOUT;
        const int w = int(std::min<long long>(PWOUT, nx - x));
        const int last = (w - 1) / GWOUT * GWOUT;
        return x + std::max(PW - 4, last + 64 - 4);
    }, xd);
    const bool ok_y = flow_axis_deps(ny, seg, n_wy, LAG, [&](int a) {
        return std::min<long long>(ny, (long long)(a + 1) * seg) + LAG;
    }, yd);
    if (!ok_x || !ok_y) return QLA_EINVAL;
    const int wx = item % n_wx, wy = item / n_wx;
    const int cx = xd[size_t(wx) * FLOW_DEPS], cy = yd[size_t(wy) * FLOW_DEPS];
    for (int k = 0; k < cx * cy; ++k) {
        const int d = yd[size_t(wy) * FLOW_DEPS + 1 + k / cx] * n_wx +
                      xd[size_t(wx) * FLOW_DEPS + 1 + k % cx];
        if (k < capacity) deps[k] = d;
    }
    *count = cx * cy;
    return QLA_OK;
}

qla_status qla_debug_flow(qla_ctx *c, long long budget_cycles, long long withhold_unit) {
    qla_status s = usable(c);
    if (s != QLA_OK) return s;
    if (budget_cycles < 0 || withhold_unit < -1)
        return fail(c, QLA_EINVAL, "qla_debug_flow: budget %lld, unit %lld", budget_cycles,
                    withhold_unit);
    c->flow_budget = budget_cycles > 0 ? budget_cycles : (1LL << 32);
    c->flow_withhold = withhold_unit;
    return QLA_OK;
}

qla_status qla_march_plan(const qla_ctx *c, int *n_items, int *n_plateau_items, int *n_sets) {
    if (!c) return QLA_EINVAL;
    const auto &u = c->uplan;
    const bool live = u.gen == c->medium_gen && u.n_uniform > 0;
    if (n_items) *n_items = live ? u.n_items : 0;
    if (n_plateau_items) *n_plateau_items = live ? u.n_uniform : 0;
    if (n_sets) *n_sets = live ? u.n_sets : 0;
    return QLA_OK;
}

const char *qla_last_error(const qla_ctx *c) { return c ? c->err.c_str() : "null context"; }

const char *qla_status_string(qla_status s) {
    switch (s) {
    case QLA_OK: return "QLA_OK";
    case QLA_EINVAL: return "QLA_EINVAL";
    case QLA_ESTATE: return "QLA_ESTATE";
    case QLA_ENOMEM: return "QLA_ENOMEM";
    case QLA_ECUDA: return "QLA_ECUDA";
    case QLA_ETIMEOUT: return "QLA_ETIMEOUT";
    case QLA_ENONFINITE: return "QLA_ENONFINITE";
    }
    return "QLA_UNKNOWN";
}

void qla_destroy(qla_ctx *c) {
    if (!c) return;
    {
        DeviceGuard dg(c->device);
        cudaStreamSynchronize(c->stream);
        if (c->owns_ws) cudaFree(c->ws);
        cudaGetLastError();
    }
    delete c;
}

}  // extern "C"
