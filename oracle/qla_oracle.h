/*
 * Plain FP64 CPU oracle for the 2D QLA step (Eq. 2e14 of arXiv 2604.21128).
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the CUDA library.
 *
 * Arrays are FP64, row-major with x fastest; state q is six contiguous
 * planes of nx*ny values (q0..q5 of Eq. 3b3).  Periodic lattice.
 */
#ifndef QLA_ORACLE_H
#define QLA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_V_ROTATION = 0, ORC_V_LITERAL = 1, ORC_V_NONE = 2, ORC_V_LCU = 3 };

void orc_angles(int nx, int ny, double delta, const double *n,
                double *theta, double *beta_x, double *beta_y);
void orc_collide_x(int nx, int ny, double *q, const double *theta, int dagger);
void orc_collide_y(int nx, int ny, double *q, const double *theta, int dagger);
void orc_stream(int nx, int ny, double *q, int comp_a, int comp_b, int axis,
                int sign, double *tmp);
void orc_U(int nx, int ny, double *q, const double *theta, int axis,
           double *tmp);
void orc_V(int nx, int ny, double *q, const double *beta_x,
           const double *beta_y, int vmode);
void orc_step(int nx, int ny, double *q, const double *theta,
              const double *beta_x, const double *beta_y, int vmode,
              double *tmp);
int orc_run(int nx, int ny, double delta, const double *n, double *q,
            long long steps, int vmode);
double orc_energy(int nx, int ny, const double *q);
void orc_fields(int nx, int ny, const double *n, const double *q, double *out);
void orc_divergence(int nx, int ny, double delta, const double *n, const double *q,
                    double *out);
void orc_divergence_aniso(int nx, int ny, double delta, const double *n_x,
                          const double *n_y, const double *q, double *out);
void orc_fields_aniso(int nx, int ny, const double *n_x, const double *n_y,
                      const double *n_z, const double *q, double *out);
void orc_angles_aniso(int nx, int ny, double delta, const double *n_x, const double *n_y,
                      const double *n_z, double *ang);
void orc3_divergence(int nx, int ny, int nz, double delta, const double *n, const double *q,
                     double *out);
int orc3_run(int nx, int ny, int nz, double delta, const double *n, double *q,
             long long steps, int vmode);
int orc_run_aniso(int nx, int ny, double delta, const double *n_x, const double *n_y,
                  const double *n_z, double *q, long long steps, int vmode);
void orc_packet(int nx, int ny, double delta, int i0, int j0, int nwx,
                int nwy, const double *n_win, double x0, double y0,
                double phi, double k0, double w, double wt, double amp,
                double *q_win);
int orc_abi_version(void);
void orc_set_threads(int n);
int orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
