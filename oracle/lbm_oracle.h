/*
 * FP64 CPU oracle of the two-component Shan-Chen D2Q9 step with wetting
 * boundary conditions (arXiv:2009.12584, Sec. 2). TEST INFRASTRUCTURE: used
 * by the tests, the smoke check and the CPU-baseline leg of the benchmark
 * only; the CUDA library neither includes nor links it.
 *
 * Arrays are row-major, n = y*nx + x, component s = 0 (A), 1 (B):
 *   f    [2][9][ny][nx]  post-streaming distributions (state at time t)
 *   rho  [2][ny][nx]     densities, 0 at solid nodes
 *   rt   [2][ny][nx]     virtual solid density of Eq. 8, non-zero only at
 *                        interface-solid nodes under ORACLE_BC_VIRTUAL_AVG
 *   F    [2][2][ny][nx]  total force per component (x, y)
 *   u    [2][ny][nx]     common velocity of Eq. 3 (x, y)
 *   mask [ny][nx]        1 = solid (phi = 1), 0 = fluid
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORACLE_BC_MARTYS_CHEN = 0, /* S = phi, Sec. 2 */
  ORACLE_BC_LLKC = 1,        /* S(x+c_i) = phi(x+c_i) rho(x), Sec. 2 */
  ORACLE_BC_VIRTUAL_AVG = 2, /* S = phi rho~, Eq. 8 */
  ORACLE_BC_CONSTANT = 3     /* S = phi rho_s, Sec. 2 (Chen et al.) */
};
enum { ORACLE_PAIR_CROSS = 0, ORACLE_PAIR_SELF = 1 };

typedef struct {
  int nx, ny;
  int periodic_x, periodic_y;
  double tau[2];     /* relaxation time per component, Eq. 1 */
  double G_AB;       /* fluid-fluid strength, Eq. 5 (G_AB = G_BA) */
  int bc;            /* ORACLE_BC_* */
  int pairing;       /* ORACLE_PAIR_*: which component's S enters Eq. 7 */
  double G_s[2];     /* G_As, G_Bs of Eq. 7 */
  double chi[2];     /* chi^A, chi^B of Eq. 8 */
  double rho_s[2];   /* constant solid densities (ORACLE_BC_CONSTANT) */
  int avg_stencil;   /* 25 (D2Q25, the paper's choice) or 9 */
} oracle_params;

/* Threads of the parallel loops (OpenMP builds; n < 1: one per core).
 * Returns the number set (1 in a serial build). Results do not depend on it. */
int oracle_set_threads(int n);
int oracle_max_threads(void);
void oracle_lattice(int *cx, int *cy, double *w, int *opp);
int oracle_d2q25(int *ex, int *ey, double *wt);
int oracle_check(const oracle_params *p, const unsigned char *mask);
void oracle_equilibrium(double rho, double ux, double uy, double *feq);
void oracle_source(double tau, double ux, double uy, double Fx, double Fy,
                   double *S);
void oracle_densities(const oracle_params *p, const unsigned char *mask,
                      const double *f, double *rho);
void oracle_interface_solid(const oracle_params *p, const unsigned char *mask,
                            unsigned char *flag);
void oracle_virtual_density(const oracle_params *p, const unsigned char *mask,
                            const double *rho, double *rt);
void oracle_forces(const oracle_params *p, const unsigned char *mask,
                   const double *rho, const double *rt, double *F);
void oracle_velocity(const oracle_params *p, const unsigned char *mask,
                     const double *f, const double *rho, const double *F,
                     double *u);
void oracle_fields(const oracle_params *p, const unsigned char *mask,
                   const double *f, double *rho, double *rt, double *F,
                   double *u);
void oracle_collide(const oracle_params *p, const unsigned char *mask,
                    const double *f, const double *rho, const double *u,
                    const double *F, double *fpost);
void oracle_stream(const oracle_params *p, const unsigned char *mask,
                   const double *fpost, double *f);
int oracle_init(const oracle_params *p, const unsigned char *mask,
                const double *rhoA, const double *rhoB, const double *ux,
                const double *uy, double *f);
int oracle_step(const oracle_params *p, const unsigned char *mask, double *f,
                int nsteps);
void oracle_mass(const oracle_params *p, const unsigned char *mask,
                 const double *f, double *out);

#ifdef __cplusplus
}
#endif
#endif
