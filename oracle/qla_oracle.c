/*
 * Plain FP64 CPU oracle for the 2D qubit lattice algorithm (QLA) of
 * Soe et al., "Quantum Computing Framework for Transient Scattering of
 * Electromagnetic Waves by Dielectric Structures" (arXiv 2604.21128).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * (the CUDA library) never links, loads or calls it, and the two share no
 * code: no header, helper, table or constant generator.
 *
 * The oracle applies the paper's operators one at a time, literally, over
 * full periodic arrays, in the order the paper writes them:
 *   Q(t + dt) = V_y V_x U_y U_x Q(t)                         (Eq. 2e14)
 * with U_x, U_y the 16-operator collide/stream products of Eq. 2e6 and
 * Eq. 2e9 (applied rightmost first), collisions C_x (Eq. 2e3) and C_y
 * (Eq. 2e8) with angles theta = delta / (4 n) (Eq. 2e4), streaming shifts of
 * Eq. 2e5, and the potential operators V_x, V_y (Eqs. 2e11-2e13).
 *
 * Readings where the paper is garbled or silent (each also listed in the
 * design notes):
 *   - the workloads are isotropic, n_x = n_y = n_z = n (Sec. V-B), so
 *     theta_0 = theta_1 = theta_2 = delta/(4n), beta_0 = beta_2, beta_1 = beta_3;
 *     the *_aniso entry points take the three indices of a diagonal tensor
 *     separately and give every pair its own angle as Eqs. 2e4, 2e8 and 2e13
 *     print them;
 *   - streaming read literally: S^{+x} q(x) <- q(x + delta);
 *   - d n / d x by the centred periodic difference (n[i+1]-n[i-1])/(2 delta);
 *   - V: default "rotation" reading (rotation by beta/2 in the planes that
 *     Eqs. 2d1-2d6 couple), or the printed shear with the q5 row sign taken
 *     from the LCU sum (Eqs. 2f1-2f4) and the q3 row of Eq. 2e12 read as
 *     sin(beta_3) q2 + cos(beta_3) q3, or no V at all (Eq. 2e10), or the
 *     linear combination of unitaries of Eqs. 2f1-2f7 emulated branch by
 *     branch exactly as printed.
 *
 * State layout: six planes q[c][j*nx + i], c = 0..5, i = x index (fastest),
 * j = y index; site (i, j) sits at (i*delta, j*delta); periodic in both axes.
 * The amplitudes are the Dyson-mapped fields of Eq. 3b3:
 *   (q0..q5) = (n E_x, n E_y, n E_z, B_x, B_y, B_z)   (c = 1).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (see build.py).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#include "qla_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

#define SITE(i, j) ((size_t)(j) * (size_t)nx + (size_t)(i))

/* ------------------------------------------------------------------ */
/* Angles of the medium: Eq. 2e4 and Eq. 2e13                         */
/* ------------------------------------------------------------------ */

void orc_angles(int nx, int ny, double delta, const double *n,
                double *theta, double *beta_x, double *beta_y)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        int jm = (j - 1 + ny) % ny, jp = (j + 1) % ny;
        for (int i = 0; i < nx; ++i) {
            int im = (i - 1 + nx) % nx, ip = (i + 1) % nx;
            double nn = n[SITE(i, j)];
            /* Eq. 2e4: theta = delta / (4 n) */
            theta[SITE(i, j)] = delta / (4.0 * nn);
            /* centred difference for the gradient of n (paper is silent) */
            double dndx = (n[SITE(ip, j)] - n[SITE(im, j)]) / (2.0 * delta);
            double dndy = (n[SITE(i, jp)] - n[SITE(i, jm)]) / (2.0 * delta);
            /* Eq. 2e13: beta = (1/n^2) (dn/dx) delta^2 */
            beta_x[SITE(i, j)] = dndx / (nn * nn) * delta * delta;
            beta_y[SITE(i, j)] = dndy / (nn * nn) * delta * delta;
        }
    }
}

/* Per-pair angles of a diagonal index tensor (n_x, n_y, n_z), eight planes
 * of N values in ang[], in this order:
 *   0: theta_1 = delta / (4 n_y)   C_x pair (q1, q5)         Eq. 2e4
 *   1: theta_2 = delta / (4 n_z)   C_x pair (q2, q4)         Eq. 2e4
 *   2: theta_0 = delta / (4 n_x)   C_y pair (q0, q5)         Eq. 2e8
 *   3: theta_2 = delta / (4 n_z)   C_y pair (q2, q3)         Eq. 2e8
 *   4: beta_0 = (d_x n_y) / n_y^2 delta^2   V_x pair (q1, q5)   Eq. 2e13
 *   5: beta_2 = (d_x n_z) / n_z^2 delta^2   V_x pair (q2, q4)
 *   6: beta_1 = (d_y n_x) / n_x^2 delta^2   V_y pair (q0, q5)
 *   7: beta_3 = (d_y n_z) / n_z^2 delta^2   V_y pair (q2, q3)
 * with the centred periodic difference for the derivatives. */
static double cdiff(const double *f, int nx, int ny, int i, int j, int axis, double delta)
{
    if (axis == 0)
        return (f[SITE((i + 1) % nx, j)] - f[SITE((i - 1 + nx) % nx, j)]) / (2.0 * delta);
    return (f[SITE(i, (j + 1) % ny)] - f[SITE(i, (j - 1 + ny) % ny)]) / (2.0 * delta);
}

void orc_angles_aniso(int nx, int ny, double delta, const double *n_x, const double *n_y,
                      const double *n_z, double *ang)
{
    size_t N = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t k = SITE(i, j);
            double ax = n_x[k], ay = n_y[k], az = n_z[k];
            ang[0 * N + k] = delta / (4.0 * ay);
            ang[1 * N + k] = delta / (4.0 * az);
            ang[2 * N + k] = delta / (4.0 * ax);
            ang[3 * N + k] = delta / (4.0 * az);
            ang[4 * N + k] = cdiff(n_y, nx, ny, i, j, 0, delta) / (ay * ay) * delta * delta;
            ang[5 * N + k] = cdiff(n_z, nx, ny, i, j, 0, delta) / (az * az) * delta * delta;
            ang[6 * N + k] = cdiff(n_x, nx, ny, i, j, 1, delta) / (ax * ax) * delta * delta;
            ang[7 * N + k] = cdiff(n_z, nx, ny, i, j, 1, delta) / (az * az) * delta * delta;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Collision operators                                                */
/* ------------------------------------------------------------------ */

/* Apply the 2x2 block [[m00, m01], [m10, m11]] of a 6x6 operator to the
 * component pair (qa, qb) at every site, with the block entries built from
 * cos/sin of the site's angle.  sa, sb select the sign pattern of the sine
 * entries: m01 = sa * sin, m10 = sb * sin. */
static void pair_rotate(int nx, int ny, double *qa, double *qb,
                        const double *angle, double angle_scale,
                        double sa, double sb)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t k = SITE(i, j);
            double a = angle[k] * angle_scale;
            double c = cos(a), s = sin(a);
            double x = qa[k], y = qb[k];
            qa[k] = c * x + sa * s * y;
            qb[k] = sb * s * x + c * y;
        }
    }
}

/* C_x of Eq. 2e3: rows q1 = cos q1 - sin q5, q5 = sin q1 + cos q5 (theta_1),
 * and q2 = cos q2 - sin q4, q4 = sin q2 + cos q4 (theta_2).  The adjoint is
 * the transpose (the sine signs swap). */
static void collide_x_pairs(int nx, int ny, double *q, const double *th15,
                            const double *th24, int dagger)
{
    size_t N = (size_t)nx * ny;
    double sa = dagger ? +1.0 : -1.0, sb = -sa;
    pair_rotate(nx, ny, q + 1 * N, q + 5 * N, th15, 1.0, sa, sb);
    pair_rotate(nx, ny, q + 2 * N, q + 4 * N, th24, 1.0, sa, sb);
}

void orc_collide_x(int nx, int ny, double *q, const double *theta, int dagger)
{
    collide_x_pairs(nx, ny, q, theta, theta, dagger);
}

/* C_y of Eq. 2e8: rows q0 = cos q0 + sin q5, q5 = -sin q0 + cos q5
 * (theta_0), and q2 = cos q2 + sin q3, q3 = -sin q2 + cos q3 (theta_2). */
static void collide_y_pairs(int nx, int ny, double *q, const double *th05,
                            const double *th23, int dagger)
{
    size_t N = (size_t)nx * ny;
    double sa = dagger ? -1.0 : +1.0, sb = -sa;
    pair_rotate(nx, ny, q + 0 * N, q + 5 * N, th05, 1.0, sa, sb);
    pair_rotate(nx, ny, q + 2 * N, q + 3 * N, th23, 1.0, sa, sb);
}

void orc_collide_y(int nx, int ny, double *q, const double *theta, int dagger)
{
    collide_y_pairs(nx, ny, q, theta, theta, dagger);
}

/* ------------------------------------------------------------------ */
/* Streaming operators: Eq. 2e5                                       */
/* ------------------------------------------------------------------ */

/* Shift one plane: new q(x, y) = old q(x + sign*delta, y) for axis 0, or
 * old q(x, y + sign*delta) for axis 1, periodic. */
static void shift_plane(int nx, int ny, double *p, int axis, int sign,
                        double *tmp)
{
    size_t N = (size_t)nx * ny;
    memcpy(tmp, p, N * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            int si = i, sj = j;
            if (axis == 0) si = ((i + sign) % nx + nx) % nx;
            else           sj = ((j + sign) % ny + ny) % ny;
            p[SITE(i, j)] = tmp[SITE(si, sj)];
        }
    }
}

/* S_{ab}^{sign, axis}: shift the components a and b, leave the others. */
void orc_stream(int nx, int ny, double *q, int comp_a, int comp_b, int axis,
                int sign, double *tmp)
{
    size_t N = (size_t)nx * ny;
    shift_plane(nx, ny, q + (size_t)comp_a * N, axis, sign, tmp);
    shift_plane(nx, ny, q + (size_t)comp_b * N, axis, sign, tmp);
}

/* ------------------------------------------------------------------ */
/* Evolution operators U_x (Eq. 2e6) and U_y (Eq. 2e9)                */
/* ------------------------------------------------------------------ */

/* One factor of the product: either a collision (C or its adjoint) or a
 * streaming shift of the pair "first" (S14 along x, S03 along y) or the pair
 * "second" (S25) by +1 or -1 cell. */
enum { OP_C = 0, OP_CDAG = 1, OP_S1P = 2, OP_S1M = 3, OP_S2P = 4, OP_S2M = 5 };

/* Eq. 2e6 read right to left, i.e. in the order the factors act on Q.
 * In the paper's left-to-right notation the product is
 *   S25+ C^ S25- C . S14- C^ S14+ C . S25- C S25+ C^ . S14+ C S14- C^
 * (C^ = adjoint), so the first factor to act is the rightmost C^.  Eq. 2e9
 * has the same pattern with S03 in place of S14. */
static const int U_SEQUENCE[16] = {
    OP_CDAG, OP_S1M, OP_C,    OP_S1P,
    OP_CDAG, OP_S2P, OP_C,    OP_S2M,
    OP_C,    OP_S1P, OP_CDAG, OP_S1M,
    OP_C,    OP_S2M, OP_CDAG, OP_S2P,
};

/* th5: angle of the pair with q5 ((q1, q5) along x, (q0, q5) along y);
 * th2: angle of the pair with q2 ((q2, q4) along x, (q2, q3) along y). */
static void U_pairs(int nx, int ny, double *q, const double *th5, const double *th2,
                    int axis, double *tmp)
{
    /* axis 0: pairs S14 = (q1, q4) and S25 = (q2, q5)   (Eq. 2e5)
     * axis 1: pairs S03 = (q0, q3) and S25 = (q2, q5)   (Eq. 2e9) */
    int f_a = (axis == 0) ? 1 : 0, f_b = (axis == 0) ? 4 : 3;
    for (int k = 0; k < 16; ++k) {
        switch (U_SEQUENCE[k]) {
        case OP_C:
        case OP_CDAG: {
            int dag = (U_SEQUENCE[k] == OP_CDAG);
            if (axis == 0) collide_x_pairs(nx, ny, q, th5, th2, dag);
            else           collide_y_pairs(nx, ny, q, th5, th2, dag);
            break;
        }
        case OP_S1P: orc_stream(nx, ny, q, f_a, f_b, axis, +1, tmp); break;
        case OP_S1M: orc_stream(nx, ny, q, f_a, f_b, axis, -1, tmp); break;
        case OP_S2P: orc_stream(nx, ny, q, 2, 5, axis, +1, tmp); break;
        case OP_S2M: orc_stream(nx, ny, q, 2, 5, axis, -1, tmp); break;
        }
    }
}

void orc_U(int nx, int ny, double *q, const double *theta, int axis,
           double *tmp)
{
    U_pairs(nx, ny, q, theta, theta, axis, tmp);
}

/* ------------------------------------------------------------------ */
/* Potential operators V_x, V_y (Eqs. 2e11-2e13)                      */
/* ------------------------------------------------------------------ */

/* Printed shear (Eq. 2e11) with the q5 row sign of the LCU sum: only the
 * rows q4 and q5 change,
 *   q4 <- -sin(b2) q2 + cos(b2) q4,   q5 <- +sin(b0) q1 + cos(b0) q5. */
static void potential_x_literal(int nx, int ny, double *q, const double *b15,
                                const double *b24)
{
    size_t N = (size_t)nx * ny;
    double *q1 = q + N, *q2 = q + 2 * N, *q4 = q + 4 * N, *q5 = q + 5 * N;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t k = SITE(i, j);
            double c2 = cos(b24[k]), s2 = sin(b24[k]);
            double c0 = cos(b15[k]), s0 = sin(b15[k]);
            q4[k] = -s2 * q2[k] + c2 * q4[k];
            q5[k] = s0 * q1[k] + c0 * q5[k];
        }
    }
}

/* Printed shear (Eq. 2e12) with the q3 row read as sin(b3) q2 + cos(b3) q3:
 *   q3 <- sin(b3) q2 + cos(b3) q3,   q5 <- -sin(b1) q0 + cos(b1) q5. */
static void potential_y_literal(int nx, int ny, double *q, const double *b05,
                                const double *b23)
{
    size_t N = (size_t)nx * ny;
    double *q0 = q, *q2 = q + 2 * N, *q3 = q + 3 * N, *q5 = q + 5 * N;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t k = SITE(i, j);
            double c3 = cos(b23[k]), s3 = sin(b23[k]);
            double c1 = cos(b05[k]), s1 = sin(b05[k]);
            q3[k] = s3 * q2[k] + c3 * q3[k];
            q5[k] = -s1 * q0[k] + c1 * q5[k];
        }
    }
}

/* Rotation reading.  The collide/stream product U_x recovers the symmetric
 * operator (1/2)[(1/n) d_x + d_x (1/n)]; what Eqs. 2d2, 2d3, 2d5, 2d6 still
 * need is a rotation at rate (1/2) (d_x n)/n^2 in the (q2, q4) and (q1, q5)
 * planes, i.e. by the angle beta/2 over one step dt = delta^2:
 *   (q2, q4) <- [[c, s], [-s, c]] (q2, q4)     angle beta_2 / 2
 *   (q1, q5) <- [[c, -s], [s, c]] (q1, q5)     angle beta_0 / 2            */
static void potential_x_rotation(int nx, int ny, double *q, const double *b15,
                                 const double *b24)
{
    size_t N = (size_t)nx * ny;
    pair_rotate(nx, ny, q + 2 * N, q + 4 * N, b24, 0.5, +1.0, -1.0);
    pair_rotate(nx, ny, q + 1 * N, q + 5 * N, b15, 0.5, -1.0, +1.0);
}

/* Same along y (Eqs. 2d1, 2d3, 2d4, 2d6):
 *   (q2, q3) <- [[c, -s], [s, c]] (q2, q3)     angle beta_3 / 2
 *   (q0, q5) <- [[c, s], [-s, c]] (q0, q5)     angle beta_1 / 2            */
static void potential_y_rotation(int nx, int ny, double *q, const double *b05,
                                 const double *b23)
{
    size_t N = (size_t)nx * ny;
    pair_rotate(nx, ny, q + 2 * N, q + 3 * N, b23, 0.5, -1.0, +1.0);
    pair_rotate(nx, ny, q + 0 * N, q + 5 * N, b05, 0.5, +1.0, -1.0);
}

/* The linear combination of unitaries of Eqs. 2f1-2f7, emulated branch by
 * branch: V = (1/2)(L1 + L2 + L3 + L4) with each L applied to the site's
 * six amplitudes as printed (full angles beta, not halved).  Its sum is the
 * printed V_x with +sin(beta_0) q1 in the q5 row, and the printed V_y with
 * the q3 row cos(beta_3) q2 + sin(beta_3) q3 (the printed L_y3, L_y4 carry
 * that row); no reading is applied here. */
static void lcu_x_site(double *v, double b0, double b2)
{
    const double c0 = cos(b0), s0 = sin(b0), c2 = cos(b2), s2 = sin(b2);
    double o[6];
    /* L_x1 = I */
    for (int r = 0; r < 6; ++r) o[r] = v[r];
    /* L_x2 (Eq. 2f2) = diag(-1, 1, 1, -1, -1, -1) */
    o[0] += -v[0]; o[1] += v[1]; o[2] += v[2]; o[3] += -v[3]; o[4] += -v[4]; o[5] += -v[5];
    /* L_x3 (Eq. 2f3) */
    o[0] += v[0];
    o[1] += c0 * v[1] - s0 * v[5];
    o[2] += c2 * v[2] + s2 * v[4];
    o[3] += v[3];
    o[4] += -s2 * v[2] + c2 * v[4];
    o[5] += s0 * v[1] + c0 * v[5];
    /* L_x4 (Eq. 2f4) */
    o[0] += v[0];
    o[1] += -c0 * v[1] + s0 * v[5];
    o[2] += -c2 * v[2] - s2 * v[4];
    o[3] += v[3];
    o[4] += -s2 * v[2] + c2 * v[4];
    o[5] += s0 * v[1] + c0 * v[5];
    for (int r = 0; r < 6; ++r) v[r] = 0.5 * o[r];
}

static void lcu_y_site(double *v, double b1, double b3)
{
    const double c1 = cos(b1), s1 = sin(b1), c3 = cos(b3), s3 = sin(b3);
    double o[6];
    /* L_y1 = I */
    for (int r = 0; r < 6; ++r) o[r] = v[r];
    /* L_y2 (Eq. 2f5) = diag(1, -1, 1, -1, -1, -1) */
    o[0] += v[0]; o[1] += -v[1]; o[2] += v[2]; o[3] += -v[3]; o[4] += -v[4]; o[5] += -v[5];
    /* L_y3 (Eq. 2f6) */
    o[0] += c1 * v[0] + s1 * v[5];
    o[1] += v[1];
    o[2] += -s3 * v[2] + c3 * v[3];
    o[3] += c3 * v[2] + s3 * v[3];
    o[4] += v[4];
    o[5] += -s1 * v[0] + c1 * v[5];
    /* L_y4 (Eq. 2f7) */
    o[0] += -c1 * v[0] - s1 * v[5];
    o[1] += v[1];
    o[2] += s3 * v[2] - c3 * v[3];
    o[3] += c3 * v[2] + s3 * v[3];
    o[4] += v[4];
    o[5] += -s1 * v[0] + c1 * v[5];
    for (int r = 0; r < 6; ++r) v[r] = 0.5 * o[r];
}

static void potential_lcu(int nx, int ny, double *q, const double *b15, const double *b24,
                          const double *b05, const double *b23)
{
    size_t N = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < (long long)N; ++k) {
        double v[6];
        for (int c = 0; c < 6; ++c) v[c] = q[(size_t)c * N + k];
        lcu_x_site(v, b15[k], b24[k]);
        lcu_y_site(v, b05[k], b23[k]);
        for (int c = 0; c < 6; ++c) q[(size_t)c * N + k] = v[c];
    }
}

/* V_x then V_y with the angle planes of orc_angles_aniso (slots 4..7). */
static void V_pairs(int nx, int ny, double *q, const double *b15, const double *b24,
                    const double *b05, const double *b23, int vmode)
{
    if (vmode == ORC_V_ROTATION) {
        potential_x_rotation(nx, ny, q, b15, b24);
        potential_y_rotation(nx, ny, q, b05, b23);
    } else if (vmode == ORC_V_LITERAL) {
        potential_x_literal(nx, ny, q, b15, b24);
        potential_y_literal(nx, ny, q, b05, b23);
    } else if (vmode == ORC_V_LCU) {
        potential_lcu(nx, ny, q, b15, b24, b05, b23);
    }
    /* ORC_V_NONE: V = I, the homogeneous step of Eq. 2e10 */
}

void orc_V(int nx, int ny, double *q, const double *beta_x,
           const double *beta_y, int vmode)
{
    V_pairs(nx, ny, q, beta_x, beta_x, beta_y, beta_y, vmode);
}

/* ------------------------------------------------------------------ */
/* Full step (Eq. 2e14) and the run loop                              */
/* ------------------------------------------------------------------ */

void orc_step(int nx, int ny, double *q, const double *theta,
              const double *beta_x, const double *beta_y, int vmode,
              double *tmp)
{
    orc_U(nx, ny, q, theta, 0, tmp);          /* U_x */
    orc_U(nx, ny, q, theta, 1, tmp);          /* U_y */
    orc_V(nx, ny, q, beta_x, beta_y, vmode);  /* V_x, then V_y */
}

/* Eq. 2e14 for a diagonal index tensor: every pair with its own angle. */
int orc_run_aniso(int nx, int ny, double delta, const double *n_x, const double *n_y,
                  const double *n_z, double *q, long long steps, int vmode)
{
    size_t N = (size_t)nx * ny;
    double *ang = malloc(8 * N * sizeof(double));
    double *tmp = malloc(N * sizeof(double));
    if (!ang || !tmp) {
        free(ang); free(tmp);
        return -1;
    }
    orc_angles_aniso(nx, ny, delta, n_x, n_y, n_z, ang);
    for (long long s = 0; s < steps; ++s) {
        U_pairs(nx, ny, q, ang + 0 * N, ang + 1 * N, 0, tmp);     /* U_x */
        U_pairs(nx, ny, q, ang + 2 * N, ang + 3 * N, 1, tmp);     /* U_y */
        V_pairs(nx, ny, q, ang + 4 * N, ang + 5 * N, ang + 6 * N, ang + 7 * N, vmode);
    }
    free(ang); free(tmp);
    return 0;
}

int orc_run(int nx, int ny, double delta, const double *n, double *q,
            long long steps, int vmode)
{
    size_t N = (size_t)nx * ny;
    double *theta = malloc(N * sizeof(double));
    double *bx = malloc(N * sizeof(double));
    double *by = malloc(N * sizeof(double));
    double *tmp = malloc(N * sizeof(double));
    if (!theta || !bx || !by || !tmp) {
        free(theta); free(bx); free(by); free(tmp);
        return -1;
    }
    orc_angles(nx, ny, delta, n, theta, bx, by);
    for (long long s = 0; s < steps; ++s)
        orc_step(nx, ny, q, theta, bx, by, vmode, tmp);
    free(theta); free(bx); free(by); free(tmp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Three dimensions (Sec. III, Eq. 3b4)                                */
/* ------------------------------------------------------------------ */

/* The paper runs its scaling tests in 3D but prints only the x and y
 * sequences.  Eq. 3b4 (with i dQ/dt = W^-1/2 M W^-1/2 Q) gives the z
 * couplings of an isotropic n:
 *   dq0/dt = -(1/n) d_z q4,   dq4/dt = -d_z (q0/n)    (like (q1, q5) along x)
 *   dq1/dt = +(1/n) d_z q3,   dq3/dt = +d_z (q1/n)    (like (q2, q4) along x)
 * so the z step is the x construction with q1 -> q0, q5 -> q4, q2 -> q1,
 * q4 -> q3: C_z rotates (q0, q4) and (q1, q3) with the sign pattern of C_x,
 * the first streamed pair is S03 (q0 and q3), the second S14 (q1 and q4),
 * in the order of Eq. 2e6; V_z rotates (q1, q3) like (q2, q4) and (q0, q4)
 * like (q1, q5) by beta_z / 2, beta_z = delta^2 (d_z n) / n^2.  The full
 * step extends Eq. 2e14: Q <- V_z V_y V_x U_z U_y U_x Q.  (A reading; the
 * tests pin it to Eq. 3b4 through the generator fit.)
 * Layout: q[c][(k * ny + j) * nx + i], k = z index; periodic in all axes. */

#define SITE3(i, j, k) (((size_t)(k) * (size_t)ny + (size_t)(j)) * (size_t)nx + (size_t)(i))

static void shift3(int nx, int ny, int nz, double *p, int axis, int sign, double *tmp)
{
    size_t N = (size_t)nx * ny * nz;
    memcpy(tmp, p, N * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int si = i, sj = j, sk = k;
                if (axis == 0)      si = ((i + sign) % nx + nx) % nx;
                else if (axis == 1) sj = ((j + sign) % ny + ny) % ny;
                else                sk = ((k + sign) % nz + nz) % nz;
                p[SITE3(i, j, k)] = tmp[SITE3(si, sj, sk)];
            }
}

static void collide3(int nx, int ny, int nz, double *q, const double *theta, int axis,
                     int dagger)
{
    size_t N = (size_t)nx * ny * nz;
    /* all three collisions are site-local: a 2D pass over N sites */
    if (axis == 0) {
        collide_x_pairs((int)N, 1, q, theta, theta, dagger);
    } else if (axis == 1) {
        collide_y_pairs((int)N, 1, q, theta, theta, dagger);
    } else {
        double sa = dagger ? +1.0 : -1.0, sb = -sa;     /* the sign pattern of C_x */
        pair_rotate((int)N, 1, q + 0 * N, q + 4 * N, theta, 1.0, sa, sb);
        pair_rotate((int)N, 1, q + 1 * N, q + 3 * N, theta, 1.0, sa, sb);
    }
}

static void U3(int nx, int ny, int nz, double *q, const double *theta, int axis, double *tmp)
{
    size_t N = (size_t)nx * ny * nz;
    /* first and second streamed pairs: x (q1,q4),(q2,q5); y (q0,q3),(q2,q5);
     * z (q0,q3),(q1,q4) */
    int f_a = axis == 0 ? 1 : 0, f_b = axis == 0 ? 4 : 3;
    int s_a = axis == 2 ? 1 : 2, s_b = axis == 2 ? 4 : 5;
    for (int k = 0; k < 16; ++k) {
        int op = U_SEQUENCE[k];
        if (op == OP_C || op == OP_CDAG) {
            collide3(nx, ny, nz, q, theta, axis, op == OP_CDAG);
            continue;
        }
        int first = op == OP_S1P || op == OP_S1M;
        int sign = (op == OP_S1P || op == OP_S2P) ? +1 : -1;
        int a = first ? f_a : s_a, b = first ? f_b : s_b;
        shift3(nx, ny, nz, q + (size_t)a * N, axis, sign, tmp);
        shift3(nx, ny, nz, q + (size_t)b * N, axis, sign, tmp);
    }
}

int orc3_run(int nx, int ny, int nz, double delta, const double *n, double *q,
             long long steps, int vmode)
{
    size_t N = (size_t)nx * ny * nz;
    double *theta = malloc(N * sizeof(double));
    double *b = malloc(3 * N * sizeof(double));
    double *tmp = malloc(N * sizeof(double));
    if (!theta || !b || !tmp || (vmode != ORC_V_ROTATION && vmode != ORC_V_NONE)) {
        free(theta); free(b); free(tmp);
        return -1;
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t s = SITE3(i, j, k);
                double nn = n[s];
                double dx = (n[SITE3((i + 1) % nx, j, k)] - n[SITE3((i + nx - 1) % nx, j, k)]) / (2.0 * delta);
                double dy = (n[SITE3(i, (j + 1) % ny, k)] - n[SITE3(i, (j + ny - 1) % ny, k)]) / (2.0 * delta);
                double dz = (n[SITE3(i, j, (k + 1) % nz)] - n[SITE3(i, j, (k + nz - 1) % nz)]) / (2.0 * delta);
                theta[s] = delta / (4.0 * nn);
                b[s] = dx / (nn * nn) * delta * delta;
                b[N + s] = dy / (nn * nn) * delta * delta;
                b[2 * N + s] = dz / (nn * nn) * delta * delta;
            }
    for (long long t = 0; t < steps; ++t) {
        U3(nx, ny, nz, q, theta, 0, tmp);
        U3(nx, ny, nz, q, theta, 1, tmp);
        U3(nx, ny, nz, q, theta, 2, tmp);
        if (vmode == ORC_V_ROTATION) {
            potential_x_rotation((int)N, 1, q, b, b);
            potential_y_rotation((int)N, 1, q, b + N, b + N);
            pair_rotate((int)N, 1, q + 1 * N, q + 3 * N, b + 2 * N, 0.5, +1.0, -1.0);
            pair_rotate((int)N, 1, q + 0 * N, q + 4 * N, b + 2 * N, 0.5, -1.0, +1.0);
        }
    }
    free(theta); free(b); free(tmp);
    return 0;
}

/* Gauss laws (Eqs. 3.1, 3.2) in 3D with centred periodic differences:
 * div B = d_x q3 + d_y q4 + d_z q5, div D = d_x (n q0) + d_y (n q1) + d_z (n q2)
 * (D = n^2 E = n q_E).  out as orc_divergence: sums of (div B)^2, of the
 * squared diagonal derivatives of B, the same two for D, max |div B|,
 * max |div D|. */
void orc3_divergence(int nx, int ny, int nz, double delta, const double *n, const double *q,
                     double *out)
{
    size_t N = (size_t)nx * ny * nz;
    const double h = 0.5 / delta;
    double sb = 0.0, gb = 0.0, sd = 0.0, gd = 0.0, mb = 0.0, md = 0.0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t xp = SITE3((i + 1) % nx, j, k), xm = SITE3((i + nx - 1) % nx, j, k);
                size_t yp = SITE3(i, (j + 1) % ny, k), ym = SITE3(i, (j + ny - 1) % ny, k);
                size_t zp = SITE3(i, j, (k + 1) % nz), zm = SITE3(i, j, (k + nz - 1) % nz);
                double bx = h * (q[3 * N + xp] - q[3 * N + xm]);
                double by = h * (q[4 * N + yp] - q[4 * N + ym]);
                double bz = h * (q[5 * N + zp] - q[5 * N + zm]);
                double dx = h * (n[xp] * q[0 * N + xp] - n[xm] * q[0 * N + xm]);
                double dy = h * (n[yp] * q[1 * N + yp] - n[ym] * q[1 * N + ym]);
                double dz = h * (n[zp] * q[2 * N + zp] - n[zm] * q[2 * N + zm]);
                double db = bx + by + bz, dd = dx + dy + dz;
                sb += db * db;
                gb += bx * bx + by * by + bz * bz;
                sd += dd * dd;
                gd += dx * dx + dy * dy + dz * dz;
                if (fabs(db) > mb) mb = fabs(db);
                if (fabs(dd) > md) md = fabs(dd);
            }
    out[0] = sb;
    out[1] = gb;
    out[2] = sd;
    out[3] = gd;
    out[4] = mb;
    out[5] = md;
}

/* ------------------------------------------------------------------ */
/* Energy (Eq. A13), fields (inverse of Eq. 3b3), initial packet       */
/* ------------------------------------------------------------------ */

/* Sum over sites and components of q_c^2: the squared norm of Q, which is
 * the total energy of Eq. A13 up to the cell area delta^2. */
double orc_energy(int nx, int ny, const double *q)
{
    size_t N = (size_t)nx * ny;
    double total = 0.0;
    for (int c = 0; c < 6; ++c) {
        double part = 0.0;
#pragma omp parallel for reduction(+ : part) schedule(static)
        for (long long k = 0; k < (long long)N; ++k)
            part += q[(size_t)c * N + k] * q[(size_t)c * N + k];
        total += part;
    }
    return total;
}

/* E = q_{0,1,2} / n and B = q_{3,4,5} (Eq. 3b3 with c = 1).  out holds six
 * planes in the order E_x, E_y, E_z, B_x, B_y, B_z. */
void orc_fields(int nx, int ny, const double *n, const double *q, double *out)
{
    orc_fields_aniso(nx, ny, n, n, n, q, out);
}

/* The same with E_x = q0 / n_x, E_y = q1 / n_y, E_z = q2 / n_z (Eq. 3b3). */
void orc_fields_aniso(int nx, int ny, const double *n_x, const double *n_y,
                      const double *n_z, const double *q, double *out)
{
    size_t N = (size_t)nx * ny;
    const double *nc[3] = {n_x, n_y, n_z};
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < (long long)N; ++k) {
        for (int c = 0; c < 3; ++c) out[c * N + k] = q[c * N + k] / nc[c][k];
        for (int c = 3; c < 6; ++c) out[c * N + k] = q[c * N + k];
    }
}

/* Gauss laws, Eqs. 3.1 and 3.2, on the lattice.  Fields vary in x and y
 * only, so div B = d_x B_x + d_y B_y and div D = d_x D_x + d_y D_y with
 * B = (q3, q4) and D = eps E = n^2 E, i.e. D_x = n q0, D_y = n q1 (Dyson
 * variables, Eq. 3b3, c = 1).  The paper does not state the discrete
 * derivative; it is read as the centred periodic difference
 * (f[i+1] - f[i-1]) / (2 delta), the same one the potential angles use.
 * out[0] = sum (div B)^2, out[1] = sum (d_x B_x)^2 + (d_y B_y)^2 (the scale
 * div B is measured against), out[2] = sum (div D)^2, out[3] the same scale
 * for D, out[4] = max |div B|, out[5] = max |div D|. */
void orc_divergence(int nx, int ny, double delta, const double *n, const double *q,
                    double *out)
{
    orc_divergence_aniso(nx, ny, delta, n, n, q, out);
}

/* D_x = n_x q0 and D_y = n_y q1 for a diagonal index tensor. */
void orc_divergence_aniso(int nx, int ny, double delta, const double *n_x,
                          const double *n_y, const double *q, double *out)
{
    size_t N = (size_t)nx * ny;
    const double *q0 = q, *q1 = q + N, *q3 = q + 3 * N, *q4 = q + 4 * N;
    double sb = 0.0, gb = 0.0, sd = 0.0, gd = 0.0, mb = 0.0, md = 0.0;
    const double h = 0.5 / delta;
    for (int j = 0; j < ny; ++j) {
        const int jp = (j + 1) % ny, jm = (j + ny - 1) % ny;
        for (int i = 0; i < nx; ++i) {
            const int ip = (i + 1) % nx, im = (i + nx - 1) % nx;
            const size_t kxp = (size_t)j * nx + ip, kxm = (size_t)j * nx + im;
            const size_t kyp = (size_t)jp * nx + i, kym = (size_t)jm * nx + i;
            const double dbx = h * (q3[kxp] - q3[kxm]);
            const double dby = h * (q4[kyp] - q4[kym]);
            const double ddx = h * (n_x[kxp] * q0[kxp] - n_x[kxm] * q0[kxm]);
            const double ddy = h * (n_y[kyp] * q1[kyp] - n_y[kym] * q1[kym]);
            const double db = dbx + dby, dd = ddx + ddy;
            sb += db * db;
            gb += dbx * dbx + dby * dby;
            sd += dd * dd;
            gd += ddx * ddx + ddy * ddy;
            if (fabs(db) > mb) mb = fabs(db);
            if (fabs(dd) > md) md = fabs(dd);
        }
    }
    out[0] = sb;
    out[1] = gb;
    out[2] = sd;
    out[3] = gd;
    out[4] = mb;
    out[5] = md;
}

/* Minimum-image offset of coordinate x from x0 on a period L, in [-L/2, L/2). */
static double min_image(double x, double x0, double L)
{
    double d = fmod(x - x0 + 0.5 * L, L);
    if (d < 0.0) d += L;
    return d - 0.5 * L;
}

/* E_z-polarised Gaussian packet (Sec. V-B), moving along the angle phi:
 *   xi  = dx cos(phi) + dy sin(phi),  eta = -dx sin(phi) + dy cos(phi)
 *   E_z = A exp(-xi^2 / w^2) cos(k0 xi) [ exp(-eta^2 / wt^2) if wt > 0 ]
 * and the plane-wave magnetic field B = n k^ x E, which in Dyson variables
 * reads q2 = n E_z, q3 = sin(phi) q2, q4 = -cos(phi) q2 (the rest zero).
 * Fills the window of nwx x nwy sites whose first site is (i0, j0) of the
 * global nx x ny lattice; n_win is the medium on that window. */
void orc_packet(int nx, int ny, double delta, int i0, int j0, int nwx,
                int nwy, const double *n_win, double x0, double y0,
                double phi, double k0, double w, double wt, double amp,
                double *q_win)
{
    size_t N = (size_t)nwx * nwy;
    double Lx = nx * delta, Ly = ny * delta;
    double cphi = cos(phi), sphi = sin(phi);
    memset(q_win, 0, 6 * N * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int jj = 0; jj < nwy; ++jj) {
        for (int ii = 0; ii < nwx; ++ii) {
            int gi = ((i0 + ii) % nx + nx) % nx;
            int gj = ((j0 + jj) % ny + ny) % ny;
            double dx = min_image(gi * delta, x0, Lx);
            double dy = min_image(gj * delta, y0, Ly);
            double xi = dx * cphi + dy * sphi;
            double eta = -dx * sphi + dy * cphi;
            double ez = amp * exp(-(xi * xi) / (w * w)) * cos(k0 * xi);
            if (wt > 0.0) ez *= exp(-(eta * eta) / (wt * wt));
            size_t k = (size_t)jj * nwx + ii;
            double q2 = n_win[k] * ez;
            q_win[2 * N + k] = q2;
            q_win[3 * N + k] = sphi * q2;
            q_win[4 * N + k] = -cphi * q2;
        }
    }
}

int orc_abi_version(void) { return 1; }

/* Thread count of the OpenMP loops (1 when built without OpenMP). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
