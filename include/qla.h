/*
 * qla.h -- C ABI of libqla, a GB300 (sm_103a) implementation of the qubit
 * lattice algorithm (QLA) for Maxwell's equations in a 2D inhomogeneous
 * scalar dielectric n(x, y), after Soe et al., arXiv 2604.21128.
 *
 * One context = one periodic nx x ny lattice of spacing delta on the current
 * CUDA device, advanced by the step of Eq. 2e14,
 *     Q(t + dt) = V_y V_x U_y U_x Q(t),      dt = delta^2 (Eq. 2e7),
 * where Q holds the six Dyson amplitudes of Eq. 3b3,
 *     (q0, q1, q2, q3, q4, q5) = (n E_x, n E_y, n E_z, c B_x, c B_y, c B_z),
 * U_x / U_y are the collide-stream products of Eqs. 2e6 / 2e9 (collisions
 * C_x Eq. 2e3, C_y Eq. 2e8 with theta = delta/(4n), Eq. 2e4; shifts Eq. 2e5)
 * and V_x / V_y the potential operators of Eqs. 2e11-2e13.
 *
 * Conventions shared by every call:
 *  - Host arrays are FP64, row-major with x fastest: element (i, j) at
 *    [j*nx + i]; site (i, j) sits at the point (i*delta, j*delta).  The
 *    lattice is periodic in x and y.  Host arrays are caller-owned and are
 *    only read or written during the call.
 *  - Every call that launches work enqueues it on the context's stream.
 *    Calls that return host data (qla_energy, qla_get_state, qla_fields)
 *    synchronise that stream; qla_step does not.
 *  - Errors are return codes; nothing is thrown across the ABI.  A CUDA
 *    error makes the context's status sticky (every later call returns
 *    QLA_ECUDA); qla_last_error() gives the text.
 *  - One context must be used from one host thread at a time.
 */
#ifndef QLA_H
#define QLA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qla_ctx qla_ctx;

typedef enum {
    QLA_OK = 0,
    QLA_EINVAL = 1,      /* bad argument (size, pointer, flag, non-finite or n <= 0) */
    QLA_ESTATE = 2,      /* call out of order (e.g. step before medium and state) */
    QLA_ENOMEM = 3,      /* device allocation failed or workspace too small */
    QLA_ECUDA = 4,       /* a CUDA call failed; the context is unusable */
    QLA_ETIMEOUT = 5,    /* a bounded device wait ran out */
    QLA_ENONFINITE = 6   /* the energy came out NaN or infinite */
} qla_status;

typedef enum { QLA_FP64 = 0, QLA_FP32 = 1 } qla_precision;

/* Context flags (bitwise or). */
enum {
    /* Evolve only q2, q3, q4 (E_z polarisation).  Exact when q0 = q1 = q5 = 0:
     * C_x couples (q1,q5),(q2,q4); C_y couples (q0,q5),(q2,q3) (Eqs. 2e3, 2e8);
     * shifts move single components; V acts in the same planes.  So the two
     * triples never mix and q0, q1, q5 stay identically zero. */
    QLA_TE_ONLY = 1u,
    /* Potential operators as printed (Eqs. 2e11-2e12, shear by the full beta
     * of Eq. 2e13), with the q5 row of V_x taken from the LCU sum
     * (Eqs. 2f1-2f4: +sin(beta_0) q1) and the q3 row of V_y read as
     * sin(beta_3) q2 + cos(beta_3) q3.  Not unitary.  Default (flag clear):
     * rotation by beta/2 in the planes (q2,q4),(q1,q5) for V_x and
     * (q2,q3),(q0,q5) for V_y, which makes Eq. 2e14 recover Eqs. 2d1-2d6
     * to O(delta^2) and the step exactly unitary. */
    QLA_POTENTIAL_LITERAL = 2u,
    /* V = I: the homogeneous-medium step of Eq. 2e10. */
    QLA_POTENTIAL_NONE = 4u,
    /* Diagonal index tensor (n_x, n_y, n_z) instead of a scalar n: the
     * workspace gains the n_x and n_y planes (and, with six planes, a wider
     * per-site record) so that qla_set_medium_tensor can give every pair its
     * own angle.  E_z contexts (QLA_TE_ONLY) see n_z only and keep every step
     * kernel; six-plane contexts step with the tile kernel. */
    QLA_ANISOTROPIC = 8u,
    /* Potential operators as the paper's linear combination of unitaries
     * (Eqs. 2f1-2f7), emulated branch by branch: each site's amplitudes are
     * sent through the four printed matrices L_1..L_4 (full angles beta) and
     * the results summed and halved.  The sum is the printed V_x (with the
     * +sin(beta_0) q5 row) and the printed V_y, whose q3 row
     * cos(beta_3) q2 + sin(beta_3) q3 overwrites B_x with n E_z wherever
     * d_y n = 0: the scheme is then unstable (the oracle's energy grows by
     * ~1e87 over 400 steps of the 256^2 ellipse workload).  For measuring
     * that, not for physics.  Excludes the two flags above; stepped by the
     * tile kernel with V applied within each launch. */
    QLA_POTENTIAL_LCU = 16u,
    /* FP64 contexts: qla_step advances with the marching kernel in
     * double-single arithmetic (each amplitude an unevaluated sum of two FP32
     * words; products exact through FMA, sums by error-free transformations;
     * cos and sin held as three FP32 words, which reproduce the FP64
     * coefficients exactly).  The state is converted in place to word pairs
     * when qla_step starts and back to FP64 when it returns, so every other
     * call sees an ordinary FP64 context.  Results differ from the native
     * FP64 kernels by rounding only (relative L2 ~1e-13 after 400 steps).
     * Not part of Eq. 2e14: an arithmetic for GPUs whose FP32 pipes are
     * much faster than their FP64 pipe.  Needs QLA_FP64, a lattice the
     * marching kernel takes (nx even, nx >= 64, ny >= 8, and the live planes
     * x ny x the padded row length (nx rounded up to 32) at most 2^32, the
     * kernel's 32-bit element offsets), a scalar medium and
     * the rotation or no-potential reading; QLA_EINVAL otherwise.  The
     * workspace gains a table of double-single coefficient records. */
    QLA_DOUBLE_SINGLE = 32u
};

/* E_z-polarised Gaussian packet (Sec. V-B): with
 *   xi  =  dx cos(angle) + dy sin(angle),  eta = -dx sin(angle) + dy cos(angle),
 * (dx, dy) the minimum-image offset of a site from (x0, y0) on the periodic
 * box, E_z = amplitude * exp(-xi^2/width^2) * cos(k0 xi), times
 * exp(-eta^2/transverse_width^2) when transverse_width > 0 (0 = planar
 * front).  B is the plane-wave field n k^ x E, so q2 = n E_z,
 * q3 = sin(angle) q2, q4 = -cos(angle) q2, and q0 = q1 = q5 = 0.
 * Lengths in physical units (cells * delta); k0 in radians per unit. */
typedef struct {
    double x0, y0, angle, k0, width, transverse_width, amplitude;
} qla_packet;

/* Bytes of device workspace a context of this shape needs (state ping-pong
 * buffers, coefficient planes, the n plane, a FP64 staging plane and the
 * reduction scratch).  0 for invalid arguments. */
size_t qla_workspace_bytes(int nx, int ny, int precision, unsigned flags);

/* Create a context.  nx, ny >= 1 with nx * ny + 4096 < 2^32 (per-site
 * record indices are 32-bit; larger lattices give QLA_EINVAL, and 0 from
 * qla_workspace_bytes); delta > 0 and finite; precision is a
 * qla_precision; cuda_stream is a cudaStream_t (NULL = legacy default
 * stream) on the current device.  workspace: device memory of at least
 * qla_workspace_bytes() bytes, 256-byte aligned, owned by the caller and
 * kept alive until qla_destroy(); or NULL, in which case the library
 * allocates (and frees) its own.  On success *out receives the context; on
 * failure *out is NULL and the return code says why. */
qla_status qla_init_grid(qla_ctx **out, int nx, int ny, double delta,
                         int precision, unsigned flags, void *cuda_stream,
                         void *workspace, size_t workspace_bytes);

/* Set the medium n(x, y) (nx*ny FP64 host values, every one finite and
 * > 0) and derive the per-site coefficients: theta = delta/(4n) (Eq. 2e4),
 * beta = delta^2 (dn/dx)/n^2 and likewise in y (Eq. 2e13), with dn/dx by
 * the centred periodic difference (n[i+1] - n[i-1])/(2 delta).  The FP64
 * angles are turned into cosine/sine coefficient planes; in FP32 mode the
 * collision coefficients are stored as two FP32 words each (value + low
 * part).  Returns QLA_EINVAL (and changes nothing) if any n is not finite
 * or not positive. */
qla_status qla_set_medium(qla_ctx *ctx, const double *n_host);

/* Set a diagonal index tensor n = diag(n_x, n_y, n_z)(x, y) (Sec. III, the
 * form in which Eqs. 2d1-2d6, 2e3-2e13 are written); three nx*ny FP64 host
 * arrays, every value finite and > 0, copied before return.  Each pair
 * takes its own angle:
 *   C_x (Eq. 2e3):  (q1, q5) theta_1 = delta/(4 n_y); (q2, q4) theta_2 = delta/(4 n_z)
 *   C_y (Eq. 2e8):  (q0, q5) theta_0 = delta/(4 n_x); (q2, q3) theta_2
 *   V_x (Eq. 2e13): (q1, q5) beta_0 = delta^2 d_x n_y / n_y^2; (q2, q4) beta_2 = delta^2 d_x n_z / n_z^2
 *   V_y:            (q0, q5) beta_1 = delta^2 d_y n_x / n_x^2; (q2, q3) beta_3 = delta^2 d_y n_z / n_z^2
 * and read-outs use E = (q0/n_x, q1/n_y, q2/n_z), D = (n_x q0, n_y q1), the
 * packet q2 = n_z E_z.  Needs a context made with QLA_ANISOTROPIC (else
 * QLA_EINVAL); on such a context qla_set_medium(n) equals
 * qla_set_medium_tensor(n, n, n).  Synchronises. */
qla_status qla_set_medium_tensor(qla_ctx *ctx, const double *n_x, const double *n_y,
                                 const double *n_z);

/* Fill the state with the packet described by *p (see qla_packet) on the
 * current medium.  QLA_ESTATE if no medium was set; QLA_EINVAL if width
 * <= 0, transverse_width < 0 or any field is not finite. */
qla_status qla_set_packet(qla_ctx *ctx, const qla_packet *p);

/* Copy a raw state in: 6*nx*ny FP64 host values, planes q0..q5 in order.
 * In QLA_TE_ONLY mode planes q0, q1, q5 must be all zero (QLA_EINVAL
 * otherwise).  In FP32 mode the values are rounded to FP32. */
qla_status qla_set_state(qla_ctx *ctx, const double *q_host);

/* Copy the state out as 6*nx*ny FP64 host values (q0..q5; zeros for the
 * planes a QLA_TE_ONLY context does not evolve).  Synchronises. */
qla_status qla_get_state(qla_ctx *ctx, double *q_host);

/* Advance n_steps >= 0 steps of Eq. 2e14 on the context's stream (returns
 * without waiting).  n_steps == 0 is a no-op; otherwise QLA_ESTATE before
 * both a medium and a state are set.  The steps run as one launch each, or
 * (FP32 E_z contexts on large lattices, see qla_set_step_kernel) as one
 * dataflow launch for the whole call; the results are the same bits. */
qla_status qla_step(qla_ctx *ctx, long long n_steps);

/* Total energy, Eq. A13 without the cell area: the sum over sites and
 * components of q_c^2, accumulated in FP64 in a fixed order (bitwise
 * reproducible for a given lattice).  Synchronises.  QLA_ENONFINITE if the
 * sum is NaN or infinite (the value is still written). */
qla_status qla_energy(qla_ctx *ctx, double *out);

/* Fields from the inverse of Eq. 3b3 (c = 1): E = (q0, q1, q2)/n,
 * B = (q3, q4, q5); each output is nx*ny FP64 host values, NULL to skip.
 * Synchronises. */
qla_status qla_fields(qla_ctx *ctx, double *Ex, double *Ey, double *Ez,
                      double *Bx, double *By, double *Bz);

/* Gauss-law monitors (Eqs. 3.1 and 3.2, which the paper tracks alongside the
 * energy).  Fields vary in x and y only, so div B = d_x B_x + d_y B_y with
 * B = (q3, q4), and div D = d_x D_x + d_y D_y with D = n^2 E = (n q0, n q1)
 * (Eq. 3b3, c = 1).  d_x f = (f[i+1] - f[i-1]) / (2 delta), periodic (the
 * paper does not state the discrete derivative).  The state is read with the
 * pending potential step applied, like every read-out.  out[6] (host):
 *   out[0] = sum (div B)^2        out[1] = sum (d_x B_x)^2 + (d_y B_y)^2
 *   out[2] = sum (div D)^2        out[3] = sum (d_x D_x)^2 + (d_y D_y)^2
 *   out[4] = max |div B|          out[5] = max |div D|
 * sqrt(out[0] / out[1]) is the relative divergence; a QLA_TE_ONLY context
 * has no in-plane D (out[2] = out[3] = out[5] = 0).  FP64 accumulation.
 * Synchronises.  QLA_ESTATE without medium and state, QLA_ENONFINITE if a
 * term is not finite. */
qla_status qla_divergence(qla_ctx *ctx, double *out);

/* Read the six amplitudes q0..q5 at `count` sites (i[k], j[k]), each
 * 0 <= i < nx, 0 <= j < ny, into out[6*k + c] (FP64; zeros for planes a
 * QLA_TE_ONLY context does not evolve).  Synchronises.  QLA_EINVAL for an
 * index out of range or count outside 0..65536. */
qla_status qla_probe(qla_ctx *ctx, int count, const int *i, const int *j, double *out);

/* ------------------------------------------------------------------------
 * Domain decomposition (Sec. V-A: the paper's code splits the lattice into
 * processor domains, each with ghost cells that are refreshed from the
 * neighbouring domains' boundary points after a step).  A sub-domain is an
 * ordinary context on its block of the global lattice plus a halo of h
 * ghost cells on every side; stepped as a periodic lattice of its own, its
 * interior stays exact for k steps when h >= 4k + 1 (U_x and U_y each reach
 * four cells per step, and the outermost ring's potential angles, Eq. 2e13,
 * use a wrapped neighbour of n), after which the halos are refilled from
 * the neighbours with the calls below.  The exchange runs in two phases --
 * x strips over the interior rows, then y strips over the full width -- so
 * the corners come along.  Contiguous buffers make each strip one send.
 * ------------------------------------------------------------------------ */

/* Bytes of a packed w x h rectangle of ctx's stored state: live planes
 * (3 for QLA_TE_ONLY, else 6) x w x h values of the storage precision (8
 * bytes for QLA_FP64 contexts, including QLA_DOUBLE_SINGLE ones, whose state
 * is FP64 between calls; 4 for QLA_FP32).  0 for a null ctx or a rectangle
 * larger than the lattice. */
size_t qla_box_bytes(const qla_ctx *ctx, int w, int h);

/* Copy the stored values of the sites (i0 .. i0+w-1, j0 .. j0+h-1) of every
 * live plane into dst_dev (device memory of qla_box_bytes(ctx, w, h) bytes,
 * layout [plane][j][i], i fastest), or back from src_dev.  The stored
 * values are the state before the last step's pending potential operator
 * (see qla_step), so boxes move only between contexts that have taken the
 * same number of steps since their states were set; the receiving context
 * applies that operator with its own coefficients.  Asynchronous on the
 * context's stream.  QLA_EINVAL for a null buffer or a rectangle outside the
 * lattice; QLA_ESTATE without a state. */
qla_status qla_pack_box(qla_ctx *ctx, int i0, int j0, int w, int h, void *dst_dev);
qla_status qla_unpack_box(qla_ctx *ctx, int i0, int j0, int w, int h, const void *src_dev);

/* Energy (Eq. A13, FP64, fixed summation order) of the sites of a
 * rectangle, e.g. a sub-domain's interior; the global energy is the FP64
 * sum over sub-domains.  Synchronises.  Errors as qla_energy, plus
 * QLA_EINVAL for a rectangle outside the lattice. */
qla_status qla_energy_box(qla_ctx *ctx, int i0, int j0, int w, int h, double *out);

/* qla_set_packet for a context that is a window of a larger periodic
 * lattice of gnx x gny sites: site (i, j) of ctx is site ((i0 + i) mod gnx,
 * (j0 + j) mod gny) of the large lattice, and the packet's minimum-image
 * distances are taken there.  With (0, 0, nx, ny) it is qla_set_packet.
 * QLA_EINVAL for bad packet fields or 0 <= i0 < gnx, 0 <= j0 < gny
 * violated; QLA_ESTATE without a medium. */
qla_status qla_set_packet_window(qla_ctx *ctx, const qla_packet *p, int i0, int j0, int gnx,
                                 int gny);

/* Step kernel.  QLA_KERNEL_AUTO picks the register-resident marching
 * kernel when the lattice suits its column layout (see
 * qla_set_march_tuning: nx a multiple of 4 for the packed-pair layout, of
 * the per-lane column count otherwise; a window of 64 or 32 x lane columns
 * no wider than nx) and ny >= 8, and the
 * shared-memory tile kernel otherwise.  QLA_KERNEL_TILE / QLA_KERNEL_MARCH
 * force one (QLA_EINVAL if the marching kernel does not support the
 * lattice, including one whose live planes exceed its 32-bit element
 * offsets: planes x ny x padded nx > 2^32).  Both compute the same operator sequence; FP64 results agree to
 * rounding order.
 * Plateau split (FP32 E_z contexts, two columns per lane, nx a multiple of
 * 4 and at least 128): the marching step runs work items whose entering
 * sites all share one record -- a plateau of n where every site's four
 * neighbours carry its n -- four columns per lane with that record's
 * collision coefficients (no index rows, no record lookups, no potential
 * step, which is the identity there); all other items take the general
 * path.  Results are bitwise those of the unsplit kernel.  The first
 * marching step after qla_set_medium or a tuning change classifies the
 * items (one small kernel and one synchronisation of the context's
 * stream), so it must not be the first call inside a stream capture.
 * QLA_KERNEL_MARCH_PLAIN = the marching kernel without the split.
 * Dataflow steps (plateau split, lattices with at least about three work
 * items per resident warp: 16384^2 at 192-row segments, 8192^2 at 64): a
 * qla_step call runs all its steps in one persistent launch (after one
 * ordinary launch for a first step with no pending potential step).  Blocks
 * take the work units of every step, four at a time, from one counter in
 * step order, and a unit of step s
 * first waits until the items whose stored sites it reads, and those that
 * read the sites it stores, have finished step s - 1 (each unit reaches
 * four sites along x and y, Eqs. 2e6 and 2e9); the per-step tail of idle
 * warps goes away and taller segments (fewer recomputed halo rows) pay.
 * Results are bitwise those of one launch per step.  Each wait gives up
 * after about two seconds of SM cycles; the next synchronising read
 * (qla_energy, qla_energy_box, qla_divergence, qla_probe, qla_fields,
 * qla_get_state) then returns QLA_ETIMEOUT and the state is undefined until
 * it is set again (steps launched before that read do no work).
 * QLA_KERNEL_MARCH_STEP = the plateau split, one launch per step;
 * QLA_KERNEL_MARCH_FLOW = dataflow steps on every lattice the plateau
 * split takes (32-row segments unless qla_set_march_tuning sets rows). */
typedef enum {
    QLA_KERNEL_AUTO = 0,
    QLA_KERNEL_TILE = 1,
    QLA_KERNEL_MARCH = 2,
    QLA_KERNEL_MARCH_PLAIN = 3,
    QLA_KERNEL_MARCH_STEP = 4,
    QLA_KERNEL_MARCH_FLOW = 5
} qla_step_kernel;
qla_status qla_set_step_kernel(qla_ctx *ctx, int kernel);

/* Segment height (rows) of the current dataflow plan into *segment_rows, 0
 * if the next steps run one launch each (or no plan is built yet). */
qla_status qla_flow_plan(const qla_ctx *ctx, int *segment_rows);

/* The items a work item of a dataflow plan waits for (host only: no
 * context, no device).  Geometry of the plan: windows of 120 stored columns
 * (nx >= 128, a multiple of 4), segments of segment_rows rows (>= 16, a
 * multiple of 4); item = segment * ceil(nx / 120) + window.  A unit of item
 * i at step s waits until every item listed here (i itself included) has
 * finished step s - 1: those whose stored sites its reads meet and those
 * whose reads meet its stored sites, per axis (a window reads 4 columns
 * left of its stored ones and up to 124 or, for its last two-column unit,
 * 60 columns past that unit's first stored column; a segment reads 4 rows
 * either side), the product of the two axes' lists.  Writes
 * min(count, capacity) item indices to deps and the full count to *count.
 * QLA_EINVAL for a geometry outside those limits. */
qla_status qla_flow_item_deps(int nx, int ny, int segment_rows, int item, int *deps,
                              int capacity, int *count);

/* Test hook for the dataflow waits (never needed in normal use):
 * budget_cycles > 0 sets each wait's limit in SM clock cycles (0 restores
 * the default 2^32, about two seconds); withhold_unit >= 0 makes the unit
 * handed out at that position of each dataflow launch (step-major: step s,
 * unit k at s * units + k) finish without counting itself, so the units
 * that depend on it wait out their limit and the next synchronising read
 * returns QLA_ETIMEOUT with no fault; -1 restores normal. */
qla_status qla_debug_flow(qla_ctx *ctx, long long budget_cycles, long long withhold_unit);

/* Energy of caller-owned device planes, allocating nothing.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory: a process whose device memory is all held
 * by another allocator (a framework's caching pool, a pre-planned serving
 * budget), or a loop that must not enter the CUDA allocator.  It computes
 * the same quantity as qla_energy -- the FP64 sum over sites and planes of
 * q^2 (Eq. A13 without the cell area) -- for planes the caller owns, with no
 * context and no workspace.
 *
 * planes: device pointer; n_planes (1..6) planes of FP64 (precision
 * QLA_FP64) or FP32 (QLA_FP32) values, element (p, j, i) at
 * planes[p * plane_stride + j * row_pitch + i] (strides in elements;
 * row_pitch >= nx, plane_stride >= row_pitch * ny).  out_dev: device pointer
 * to one double that receives the sum.  The work is enqueued on cuda_stream
 * (NULL = legacy default stream) on the current device and the call returns
 * without waiting.
 *
 * The reduction's partial sums live in one fixed device array inside the
 * library, QLA_NOALLOC_MAX_PARTIALS doubles (128 KiB), which every GPU that
 * loads the library holds until the process exits.  One partial covers
 * QLA_NOALLOC_SITES_PER_PARTIAL sites, so lattices of more than
 * QLA_NOALLOC_MAX_PARTIALS * QLA_NOALLOC_SITES_PER_PARTIAL = 2^28 sites
 * (16384 x 16384) are rejected with QLA_EINVAL before anything runs.  Every
 * call overwrites the partials it reads, so nothing carries over from the
 * previous call; but all calls share that array, so calls whose work
 * overlaps on the GPU (concurrent streams, or several host threads) race and
 * must be ordered by the caller.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  The result is bitwise reproducible for a given size
 * and agrees with qla_energy to rounding order.
 * Errors: QLA_EINVAL for a null pointer or a bad size/precision/stride,
 * QLA_ECUDA if the lookup or a launch fails, or if a CUDA error of earlier
 * work on this thread is still pending when the call starts (nothing is
 * launched then, and that error is left in place for its owner to read). */
#define QLA_NOALLOC_MAX_PARTIALS 16384
#define QLA_NOALLOC_SITES_PER_PARTIAL 16384
qla_status qla_energy_noalloc(const void *planes, int precision, int n_planes, int nx,
                              int ny, long long row_pitch, long long plane_stride,
                              void *cuda_stream, double *out_dev);

/* Tuning of the marching kernel: lane_cols = the column layout of a warp's
 * window (0 = library choice).  For FP32 E_z contexts: 1 = packed pairs
 * (each lane holds two columns 32 apart and rotates both with FP32x2
 * instructions; 64-column windows; nx a multiple of 4), 5 = packed pairs
 * with U_x of row J + 1 interleaved with U_y of row J (two independent
 * chains per warp), 2 or 4 = that many adjacent columns per lane (scalar
 * FP32; 2 is the default).  Other contexts always use 2.  rows = rows per work
 * item (0 = chosen from the occupancy so one wave of items fills the GPU;
 * else rounded up to a multiple of 4).  Results do not depend on either.
 * QLA_EINVAL for other values. */
qla_status qla_set_march_tuning(qla_ctx *ctx, int lane_cols, int rows);

/* ------------------------------------------------------------------------
 * Batched lattices.  A batch holds `count` independent periodic lattices
 * (sizes nx[k] x ny[k], common delta, precision and flags) in one workspace
 * and advances all of them together with one persistent kernel launch per
 * chunk of steps: every warp of a co-resident (cooperative) grid takes work
 * items -- a column window and row segment of some lattice -- and the grid
 * synchronises between steps with a barrier whose wait is bounded.
 * Instance k is an ordinary context (qla_batch_instance): set its medium and
 * packet or state, read its energy, fields or probes with the qla_* calls.
 * ------------------------------------------------------------------------ */
typedef struct qla_batch qla_batch;

/* Workspace bytes for a batch (0 for invalid arguments). */
size_t qla_batch_workspace_bytes(int count, const int *nx, const int *ny, int precision,
                                 unsigned flags);

/* Create a batch of `count` >= 1 lattices; every nx[k] must be a multiple
 * of 4 and >= 128, every ny[k] >= 8, and the live planes (3 with
 * QLA_TE_ONLY, else 6) x ny[k] x nx[k] rounded up to 32 at most 2^32 (the
 * marching kernel's requirements: 32-bit element offsets).
 * workspace / workspace_bytes / cuda_stream as for qla_init_grid. */
qla_status qla_batch_create(qla_batch **out, int count, const int *nx, const int *ny,
                            double delta, int precision, unsigned flags, void *cuda_stream,
                            void *workspace, size_t workspace_bytes);

/* The context of instance k (owned by the batch; do not destroy it). */
qla_ctx *qla_batch_instance(qla_batch *b, int k);

/* Advance every instance by n_steps >= 0 steps of Eq. 2e14: persistent
 * launches of at most QLA_BATCH_CHUNK steps each, enqueued on the batch's
 * stream.  Every instance must have a medium and a state.  Returns
 * QLA_ETIMEOUT (and leaves the states undefined) if a grid barrier's bounded
 * wait ran out; the check synchronises the stream after the last chunk. */
#define QLA_BATCH_CHUNK 1000
qla_status qla_batch_step(qla_batch *b, long long n_steps);

/* Run n_steps steps reading every instance's energy every `every` steps:
 * the whole sequence (persistent step launches and batched energy
 * reductions) is captured once as a CUDA graph and replayed.  energies
 * receives (n_steps / every) * count doubles, row r holding all instances'
 * energies after (r + 1) * every steps.  n_steps must be a multiple of every.
 * Synchronises. */
qla_status qla_batch_run(qla_batch *b, long long n_steps, long long every, double *energies);

/* Energy (as qla_energy) of every instance into out[0..count). Synchronises. */
qla_status qla_batch_energy(qla_batch *b, double *out);

/* Autotuner: time each candidate (lane layout in {1, 2} for FP32 E_z
 * batches -- packed pairs or two adjacent columns per lane, see
 * qla_set_march_tuning -- and rows per work item in {64, 128, 256}) on
 * `trial_steps` real steps and keep the fastest.
 * The states advance by 6 * trial_steps steps, as if qla_batch_step had
 * been called.  *chosen_lane_cols / *chosen_rows (may be NULL) receive the
 * choice. */
qla_status qla_batch_autotune(qla_batch *b, int trial_steps, int *chosen_lane_cols,
                              int *chosen_rows);

/* Tiling used by later qla_batch_step / qla_batch_run calls (as for
 * qla_set_march_tuning; 0 = library choice). */
qla_status qla_batch_set_tuning(qla_batch *b, int lane_cols, int rows);

/* Test hook for the bounded grid barrier (never needed in normal use):
 * budget_cycles > 0 sets each barrier wait's limit in SM clock cycles
 * (default 2^31, about one second); skip_block >= 0 makes that block skip
 * its arrival at the first barrier, so every other block's wait runs out
 * and the step returns QLA_ETIMEOUT with no fault.  -1 restores normal. */
qla_status qla_batch_debug_barrier(qla_batch *b, long long budget_cycles, int skip_block);

/* Kernel launches enqueued by the batch (persistent and energy). */
long long qla_batch_launch_count(const qla_batch *b);

const char *qla_batch_last_error(const qla_batch *b);

/* Free the batch (and its workspace if the library allocated it). */
void qla_batch_destroy(qla_batch *b);

/* ------------------------------------------------------------------------
 * Learned surrogate.  Not part of the paper's method: a convolutional
 * operator that advances an FP32 E_z lattice (rotation reading) K steps at
 * once, trained on trajectories this library computes, with plain QLA as
 * the fallback and arbiter.  Network: five levels of widths 32, 64, 128, 256,
 * 256; 3x3 periodic convolutions, leaky ReLU 0.1, 2x2 average pooling,
 * nearest 2x upsampling with additive skips; BF16 weights and activations,
 * FP32 accumulation on the tensor cores, FP32 master weights and Adam.
 * The convolutions' device waits are bounded: a wait that runs out makes
 * the next synchronising call (surr_loss_grad, surr_train_step,
 * surr_advance) return QLA_ETIMEOUT.
 * Inputs per site (features, FP32 [h][w][6]): q2, q3, q4, n - 1.5,
 * 4 dn/dx, 4 dn/dy; output ([h][w][3]): the change of q2, q3, q4.
 * ------------------------------------------------------------------------ */
typedef struct surr_net surr_net;

/* Device workspace bytes for a network on h x w lattices (multiples of 16)
 * and batches of up to max_batch; 0 for invalid sizes. */
size_t surr_workspace_bytes(int height, int width, int max_batch);

/* Create a network with seeded initial weights in a caller-owned device
 * workspace (256-byte aligned, kept alive until surr_destroy). */
qla_status surr_create(surr_net **out, int height, int width, int max_batch,
                       unsigned long long seed, void *cuda_stream, void *workspace,
                       size_t workspace_bytes);

/* Number of parameters, and their host copy: per convolution (10 of them,
 * encoder levels 0..4, decoder levels 3..0, output) the weights as
 * (cout, cin, 3, 3) then the biases (cout), real channel counts (the first
 * convolution has cin = 6, the last cout = 3). */
long long surr_param_count(const surr_net *n);
qla_status surr_get_params(surr_net *n, float *host);
qla_status surr_set_params(surr_net *n, const float *host);

/* Forward pass on B samples: feat_dev [B][h][w][6] -> out_dev [B][h][w][3]
 * (device FP32).  Asynchronous on the network's stream. */
qla_status surr_forward(surr_net *n, const float *feat_dev, int B, float *out_dev);

/* Mean-square loss against target_dev [B][h][w][3] and its gradient with
 * respect to every parameter (grad_host, surr_param_count floats, same
 * layout as surr_get_params; NULL to skip).  Synchronises. */
qla_status surr_loss_grad(surr_net *n, const float *feat_dev, const float *target_dev, int B,
                          double *loss, float *grad_host);

/* One Adam step (beta 0.9, 0.999, eps 1e-8) at learning rate lr. */
qla_status surr_train_step(surr_net *n, const float *feat_dev, const float *target_dev, int B,
                           float lr, double *loss);

/* Features of a context's current state into feat_dev ([ny][nx][6]). */
qla_status surr_features(qla_ctx *ctx, float *feat_dev);

/* Advance `windows` windows of K steps: each window the network proposes
 * the state K steps on; it is accepted only if the energy changes by at
 * most energy_tol (relative; the exact step conserves it) and the discrete
 * divergence of B changes by at most div_tol relative to |grad B| (the exact
 * dynamics keep div B constant); otherwise the window is recomputed with
 * qla_step(ctx, K).  scratch_dev: 12 * nx * ny floats.  *accepted receives
 * the number of accepted windows; energies (may be NULL) the energy after
 * each window.  The network must have been created for nx x ny. */
qla_status surr_advance(qla_ctx *ctx, surr_net *n, int windows, int K, double energy_tol,
                        double div_tol, float *scratch_dev, int *accepted, double *energies);

/* Text of the last error on this network ("" if none); valid until the
 * next call on it. */
const char *surr_last_error(const surr_net *n);
/* Wait for the network's stream, then free its host-side handle; the
 * device workspace stays the caller's. */
void surr_destroy(surr_net *n);

/* The network's two contraction kernels on their own (device pointers,
 * NHWC, channel counts multiples of 32), for tests:
 *   out[p][co] = sum_{tap, ci} w[co][tap][ci] in[p + shift(tap)][ci]
 *   dw[co][tap][ci] = sum_p dz[p][co] in[p + shift(tap)][ci]
 * with tap = 3 (dy + 1) + (dx + 1), shifts periodic in y and x; in, w, dz
 * BF16, out and dw FP32; part holds splits * cout * 9 * cin floats. */
qla_status surr_conv3x3_raw(const void *in_bf16, int B, int H, int W, int cin,
                            const void *w_bf16, int cout, float *out_f32, void *cuda_stream);
qla_status surr_weight_grad_raw(const void *dz_bf16, const void *in_bf16, int B, int H, int W,
                                int cout, int cin, int splits, float *part, float *dw_f32,
                                void *cuda_stream);

/* Test hook for the bounded waits: while on is non-zero, one CTA of every
 * gather-form tensor-core convolution waits for an mbarrier phase that never
 * completes, gives up after 2 s of wall time, skips its output and raises
 * the error flag, so surr_conv3x3_raw returns QLA_ETIMEOUT (and the
 * network's next synchronising call would).  No fault and no hang: the other
 * CTAs finish, the stalled one frees its tensor memory and returns. */
qla_status surr_test_stall_conv(int on);

/* ------------------------------------------------------------------------
 * Three dimensions.  The paper runs its scaling tests with a 3D code whose z
 * sequence it does not print; Eq. 3b4 (i dQ/dt = W^-1/2 M W^-1/2 Q) fixes
 * the z couplings of an isotropic n:
 *   dq0/dt = -(1/n) d_z q4,  dq4/dt = -d_z(q0/n);  dq1/dt = (1/n) d_z q3,
 *   dq3/dt = d_z(q1/n)
 * so U_z is the construction of Eq. 2e6 with C_z rotating (q0, q4) and
 * (q1, q3) by +theta (the sign pattern of C_x), S03 (q0, q3) as the first
 * and S14 (q1, q4) as the second streamed pair; V_z rotates (q1, q3) and
 * (q0, q4) by beta_z / 2 (beta_z = delta^2 d_z n / n^2) as V_x rotates
 * (q2, q4) and (q1, q5); the step is Q <- V_z V_y V_x U_z U_y U_x Q.
 * All six planes evolve (the E_z triple does not decouple in 3D).
 * Lattice nx x ny x nz, periodic, site (i, j, k) at host index
 * (k * ny + j) * nx + i; ny, nz <= 65535.  Flags: 0 (rotation reading) or
 * QLA_POTENTIAL_NONE, optionally with QLA_DOUBLE_SINGLE (FP64 contexts
 * whose nx is even and >= 64 and ny >= 8: qla3_step converts the state in
 * place, runs the slices and column kernels in double-single arithmetic
 * whatever qla3_set_step_kernel chose, and converts back); others give
 * QLA_EINVAL.  Same status conventions and stream semantics as the 2D
 * context.
 * ------------------------------------------------------------------------ */
typedef struct qla3_ctx qla3_ctx;

/* Device workspace bytes for a 3D context; 0 for invalid arguments. */
size_t qla3_workspace_bytes(int nx, int ny, int nz, int precision, unsigned flags);

/* Create a 3D context; workspace as for qla_init_grid (256-byte aligned,
 * caller-owned, or NULL to let the library allocate it). */
qla_status qla3_init(qla3_ctx **out, int nx, int ny, int nz, double delta, int precision,
                     unsigned flags, void *cuda_stream, void *workspace,
                     size_t workspace_bytes);

/* Medium n(x, y, z): nx*ny*nz FP64 host values, finite and > 0, copied
 * before return; theta = delta/(4n) and beta_x, beta_y, beta_z by centred
 * periodic differences (Eqs. 2e4, 2e13 extended to z).  Synchronises. */
qla_status qla3_set_medium(qla3_ctx *ctx, const double *n_host);

/* Raw Dyson amplitudes in or out: one host array of 6 * nx*ny*nz FP64
 * values, plane c at offset c * nx*ny*nz (caller-owned; finite on input).
 * Synchronise. */
qla_status qla3_set_state(qla3_ctx *ctx, const double *q_host);
qla_status qla3_get_state(qla3_ctx *ctx, double *q_host);

/* The E_z packet of qla_set_packet (Sec. V-B), uniform along z: every
 * slice holds the 2D packet on the current medium (q2 = n E_z,
 * q3 = sin(angle) q2, q4 = -cos(angle) q2, q0 = q1 = q5 = 0).  QLA_ESTATE
 * without a medium; QLA_EINVAL as for qla_set_packet. */
qla_status qla3_set_packet(qla3_ctx *ctx, const qla_packet *p);

/* Advance n_steps steps (see qla3_set_step_kernel for the launches);
 * asynchronous on the context's stream.  QLA_ESTATE without
 * medium and state. */
qla_status qla3_step(qla3_ctx *ctx, long long n_steps);

/* Sum of q^2 over sites and planes (Eq. A13 without the cell volume),
 * FP64.  Synchronises; QLA_ENONFINITE if not finite. */
qla_status qla3_energy(qla3_ctx *ctx, double *out);

/* Step kernel (results agree bit for bit: every kernel applies the same
 * operations in the same order per site):
 *   3: one launch per axis (U_x; U_y; U_z then V), shared-memory layers;
 *   1: one launch marching along z (U_x, U_y in shared memory per plane,
 *      U_z as a register pipeline, then V): a third of the data of 3 but
 *      slower on the GPUs measured, its per-plane barriers dominate;
 *   2: two launches: the 2D marching kernel on every z slice (U_x, U_y in
 *      registers) and a column pipeline along z (U_z, then V); needs nx
 *      even and >= 64, ny >= 8 and 6 * nz*ny*pitch < 2^32, else runs 3;
 *   0 (default): 2 for FP32 (1.8x kernel 3 at 256^3), 3 for FP64 (FP64-pipe
 *      bound, where kernel 2's window halo costs more than it saves).
 * QLA_EINVAL for other values. */
qla_status qla3_set_step_kernel(qla3_ctx *ctx, int kernel);

/* Gauss-law monitors in 3D (Eqs. 3.1, 3.2; the paper monitors them in its
 * 3D runs): div B = d_x q3 + d_y q4 + d_z q5, div D = d_x(n q0) + d_y(n q1)
 * + d_z(n q2), centred periodic differences; out[6] as qla_divergence
 * (sums of (div B)^2, of (d_x B_x)^2 + (d_y B_y)^2 + (d_z B_z)^2, the same
 * two for D, max |div B|, max |div D|), FP64.  Synchronises; QLA_ESTATE
 * without medium and state, QLA_ENONFINITE if a term is not finite. */
qla_status qla3_divergence(qla3_ctx *ctx, double *out);

/* Kernel launches enqueued by this context since creation (diagnostics; a
 * double-single step counts its per-triple slices launches separately). */
long long qla3_launch_count(const qla3_ctx *ctx);
/* Text of the last error on this context ("" if none); valid until the next
 * call on the context. */
const char *qla3_last_error(const qla3_ctx *ctx);
/* Free the context (and its workspace if the library allocated it). */
void qla3_destroy(qla3_ctx *ctx);

/* Kernel launches enqueued by this context since creation (diagnostics; a
 * six-plane double-single step is two launches, one per decoupled triple). */
long long qla_launch_count(const qla_ctx *ctx);

/* The plateau plan of the FP32 E_z marching step (see qla_set_step_kernel),
 * as built for the current medium and tuning by the last marching step:
 * work items (128-column windows x row segments) per step, items run on the
 * plateau path, and distinct plateau records among them.  All zero when no
 * plan is in use (other contexts, another kernel, no plateau item, or no
 * step since the medium or the tuning changed).  Any output pointer may be
 * NULL.  QLA_EINVAL for a null ctx. */
qla_status qla_march_plan(const qla_ctx *ctx, int *n_items, int *n_plateau_items, int *n_sets);

/* Text of the last error on this context ("" if none); valid until the next
 * call on the context.  qla_status_string() names a status code. */
const char *qla_last_error(const qla_ctx *ctx);
const char *qla_status_string(qla_status s);

/* Free the context (and the workspace if the library allocated it).
 * Synchronises the context's stream first.  NULL is a no-op. */
void qla_destroy(qla_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* QLA_H */
