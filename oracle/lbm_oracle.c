/*
 * FP64 CPU oracle for the two-component Shan-Chen D2Q9 lattice-Boltzmann step
 * with wetting boundary conditions (Coelho, Moura, Telo da Gama, Araujo,
 * "Wetting boundary conditions for multicomponent pseudopotential lattice
 * Boltzmann", arXiv:2009.12584, Sec. 2).
 *
 * TEST INFRASTRUCTURE. This file is the plain, slow reference that the CUDA
 * library is checked against. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it; the product library never links,
 * includes or calls it, and it shares no code with the CUDA sources.
 *
 * Everything is double precision, plain loops, one pass per equation, in the
 * order the paper states the method. No blocking, fusion or reordering.
 * When built with OpenMP, the loops over nodes (or rows of nodes) run in
 * parallel: every node's value is computed by one thread with the same
 * arithmetic in the same order, so the results are bit for bit those of a
 * serial build. The mass sum stays serial (its order fixes its rounding).
 *
 * Storage: f[(s*9 + i)*N + n], s = component (0 = A, 1 = B), i = D2Q9
 * direction, n = y*nx + x. The stored state is the post-streaming
 * distribution at time t (what Eq. 1's left-hand side produces). Solid nodes
 * hold zeros and are never read.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *  - Eq. 8 weights the average by phi, the solid indicator, but the text
 *    asks for the average density of the fluid neighbours: the fluid
 *    indicator (1 - phi) is used in numerator and denominator.
 *  - Eq. 7 pairs the force on sigma with S of the other component (sigma
 *    bar). That is the default ("cross"); the alternative reading that pairs
 *    it with S of sigma itself ("self") is a flag.
 *  - On a non-periodic axis, nodes outside the box count as solid; a fluid
 *    node may not touch such a border (the paper puts explicit walls at the
 *    borders, Sec. 3.1), and oracle_check rejects masks where one does.
 *  - Initial state: f = f^eq(rho, u) at fluid nodes (the paper is silent).
 */
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "lbm_oracle.h"

/* D2Q9 quadrature, Sec. 2 (text after Eq. 1): the rest velocity, the four
 * axis neighbours (|c|^2 = 1, w = 1/9) and the four diagonal neighbours
 * (|c|^2 = 2, w = 1/36); c_s^2 = 1/3. */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

/* Index of -c_i (halfway bounce-back reverses a population). */
static int opposite(int i) {
  for (int j = 0; j < 9; ++j)
    if (CX[j] == -CX[i] && CY[j] == -CY[i]) return j;
  return -1;
}

/* D2Q25 weight by |c|^2, the case list printed after Eq. 8. The 24 vectors
 * are all (dx, dy) with |dx|, |dy| <= 2 except (0, 0). */
static double d2q25_weight(int dx, int dy) {
  int r2 = dx * dx + dy * dy;
  switch (r2) {
    case 1: return 4.0 / 21.0;
    case 2: return 4.0 / 45.0;
    case 4: return 1.0 / 60.0;
    case 5: return 2.0 / 315.0;
    case 8: return 1.0 / 5040.0;
    default: return 0.0;
  }
}

/* Node index of (x + dx, y + dy), wrapping periodic axes; -1 outside a
 * non-periodic box. */
static long neighbour(const oracle_params *p, int x, int y, int dx, int dy) {
  int xx = x + dx, yy = y + dy;
  if (p->periodic_x) {
    xx = ((xx % p->nx) + p->nx) % p->nx;
  } else if (xx < 0 || xx >= p->nx) {
    return -1;
  }
  if (p->periodic_y) {
    yy = ((yy % p->ny) + p->ny) % p->ny;
  } else if (yy < 0 || yy >= p->ny) {
    return -1;
  }
  return (long)yy * p->nx + xx;
}

/* phi of Sec. 2: 1 for solid (or outside a non-periodic box), 0 for fluid. */
static int phi(const unsigned char *mask, long n) {
  return (n < 0 || mask[n] != 0) ? 1 : 0;
}

int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n < 1) n = omp_get_num_procs();
  omp_set_num_threads(n);
  return n;
#else
  (void)n;
  return 1;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_lattice(int *cx, int *cy, double *w, int *opp) {
  for (int i = 0; i < 9; ++i) {
    cx[i] = CX[i];
    cy[i] = CY[i];
    w[i] = W9[i];
    opp[i] = opposite(i);
  }
}

int oracle_d2q25(int *ex, int *ey, double *wt) {
  int k = 0;
  for (int dy = -2; dy <= 2; ++dy)
    for (int dx = -2; dx <= 2; ++dx) {
      if (dx == 0 && dy == 0) continue;
      ex[k] = dx;
      ey[k] = dy;
      wt[k] = d2q25_weight(dx, dy);
      ++k;
    }
  return k;
}

int oracle_check(const oracle_params *p, const unsigned char *mask) {
  if (p->nx < 1 || p->ny < 1) return 1;
  if (p->tau[0] <= 0.5 || p->tau[1] <= 0.5) return 1;
  if (p->bc < ORACLE_BC_MARTYS_CHEN || p->bc > ORACLE_BC_CONSTANT) return 1;
  for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) {
      long n = (long)y * p->nx + x;
      if (mask[n]) continue;
      if (!p->periodic_x && (x == 0 || x == p->nx - 1)) return 2;
      if (!p->periodic_y && (y == 0 || y == p->ny - 1)) return 2;
    }
  return 0;
}

/* Eq. 2: second-order Hermite equilibrium of one component. */
void oracle_equilibrium(double rho, double ux, double uy, double *feq) {
  double u2 = ux * ux + uy * uy;
  for (int i = 0; i < 9; ++i) {
    double cu = CX[i] * ux + CY[i] * uy;
    feq[i] = rho * W9[i] *
             (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - u2 / (2.0 * CS2));
  }
}

/* Eq. 4: Guo source term of one component with relaxation time tau. */
void oracle_source(double tau, double ux, double uy, double Fx, double Fy,
                   double *S) {
  for (int i = 0; i < 9; ++i) {
    double cu = CX[i] * ux + CY[i] * uy;
    double ax = CX[i] / CS2 * (1.0 + cu / CS2) - ux / CS2;
    double ay = CY[i] / CS2 * (1.0 + cu / CS2) - uy / CS2;
    S[i] = W9[i] * (1.0 - 1.0 / (2.0 * tau)) * (ax * Fx + ay * Fy);
  }
}

/* Density of each component at fluid nodes, rho^sigma = sum_i f_i^sigma
 * (Eq. 3, right); zero at solid nodes. */
void oracle_densities(const oracle_params *p, const unsigned char *mask,
                      const double *f, double *rho) {
  long N = (long)p->nx * p->ny;
  for (int s = 0; s < 2; ++s)
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
      double r = 0.0;
      if (!mask[n])
        for (int i = 0; i < 9; ++i) r += f[(s * 9 + i) * N + n];
      rho[s * N + n] = r;
    }
}

/* Interface-solid nodes: solid nodes with at least one fluid neighbour in
 * the D2Q9 first belt (Sec. 2, last paragraph; Sec. 3.2). */
void oracle_interface_solid(const oracle_params *p, const unsigned char *mask,
                            unsigned char *flag) {
#pragma omp parallel for schedule(static)
  for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) {
      long n = (long)y * p->nx + x;
      int any_fluid = 0;
      if (mask[n])
        for (int i = 1; i < 9; ++i)
          if (!phi(mask, neighbour(p, x, y, CX[i], CY[i]))) any_fluid = 1;
      flag[n] = (unsigned char)any_fluid;
    }
}

/* Eq. 8: virtual solid density at interface-solid nodes, chi^sigma times the
 * weighted mean density of the fluid neighbours. The weights are the D2Q25
 * set (the paper's choice) or, with avg_stencil == 9, the D2Q9 set. Zero at
 * every other node. */
void oracle_virtual_density(const oracle_params *p, const unsigned char *mask,
                            const double *rho, double *rt) {
  long N = (long)p->nx * p->ny;
  unsigned char *iface = (unsigned char *)malloc((size_t)N);
  oracle_interface_solid(p, mask, iface);
  int reach = (p->avg_stencil == 9) ? 1 : 2;
  for (int s = 0; s < 2; ++s)
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        long n = (long)y * p->nx + x;
        rt[s * N + n] = 0.0;
        if (!iface[n]) continue;
        double num = 0.0, den = 0.0;
        for (int dy = -reach; dy <= reach; ++dy)
          for (int dx = -reach; dx <= reach; ++dx) {
            if (dx == 0 && dy == 0) continue;
            double wj;
            if (p->avg_stencil == 9) {
              wj = (dx * dx + dy * dy == 1) ? 1.0 / 9.0 : 1.0 / 36.0;
            } else {
              wj = d2q25_weight(dx, dy);
            }
            long m = neighbour(p, x, y, dx, dy);
            double fluid = 1.0 - phi(mask, m);
            if (fluid == 0.0) continue;
            num += wj * rho[s * N + m] * fluid;
            den += wj * fluid;
          }
        rt[s * N + n] = p->chi[s] * num / den;
      }
  free(iface);
}

/* Solid pseudopotential S^c(x + c_i) seen from fluid node n, for the four
 * schemes of Sec. 2: Martys-Chen S = phi; Li-Luo-Kang-Chen S(x + c_i) =
 * phi(x + c_i) rho^c(x); improved virtual density S = phi rho~^c (Eq. 8);
 * Chen et al. constant S = phi rho_s^c. Only called for solid x + c_i. */
static double solid_potential(const oracle_params *p, int c, long n, long m,
                              const double *rho, const double *rt) {
  long N = (long)p->nx * p->ny;
  switch (p->bc) {
    case ORACLE_BC_MARTYS_CHEN: return 1.0;
    case ORACLE_BC_LLKC: return rho[c * N + n];
    case ORACLE_BC_VIRTUAL_AVG: return rt[c * N + m];
    case ORACLE_BC_CONSTANT: return p->rho_s[c];
  }
  return 0.0;
}

/* Total interaction force on each component at fluid nodes: the Shan-Chen
 * force of Eq. 5 summed over fluid neighbours only, plus the adhesion force
 * of Eq. 7. psi = rho, Delta t = 1. F[(s*2 + d)*N + n], d = 0 (x), 1 (y). */
void oracle_forces(const oracle_params *p, const unsigned char *mask,
                   const double *rho, const double *rt, double *F) {
  long N = (long)p->nx * p->ny;
  for (int s = 0; s < 2; ++s) {
    int sb = 1 - s;                       /* sigma bar */
    int cs = (p->pairing == ORACLE_PAIR_SELF) ? s : sb;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        long n = (long)y * p->nx + x;
        double fsc_x = 0.0, fsc_y = 0.0, fs_x = 0.0, fs_y = 0.0;
        if (!mask[n]) {
          for (int i = 1; i < 9; ++i) {
            long m = neighbour(p, x, y, CX[i], CY[i]);
            if (!phi(mask, m)) {
              /* Eq. 5, fluid neighbours only */
              fsc_x += W9[i] * rho[sb * N + m] * CX[i];
              fsc_y += W9[i] * rho[sb * N + m] * CY[i];
            } else {
              /* Eq. 7 */
              double S = solid_potential(p, cs, n, m, rho, rt);
              fs_x += W9[i] * S * CX[i];
              fs_y += W9[i] * S * CY[i];
            }
          }
          fsc_x *= -rho[s * N + n] * p->G_AB;
          fsc_y *= -rho[s * N + n] * p->G_AB;
          fs_x *= -rho[s * N + n] * p->G_s[s];
          fs_y *= -rho[s * N + n] * p->G_s[s];
        }
        F[(s * 2 + 0) * N + n] = fsc_x + fs_x;
        F[(s * 2 + 1) * N + n] = fsc_y + fs_y;
      }
  }
}

/* Eq. 3: common velocity u^eq = sum_sigma (sum_i f_i c_i + F/2) / rho with
 * rho = rho^A + rho^B. u[d*N + n]. Zero at solid nodes. */
void oracle_velocity(const oracle_params *p, const unsigned char *mask,
                     const double *f, const double *rho, const double *F,
                     double *u) {
  long N = (long)p->nx * p->ny;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; ++n) {
    double jx = 0.0, jy = 0.0;
    if (!mask[n]) {
      for (int s = 0; s < 2; ++s) {
        for (int i = 0; i < 9; ++i) {
          jx += f[(s * 9 + i) * N + n] * CX[i];
          jy += f[(s * 9 + i) * N + n] * CY[i];
        }
        jx += F[(s * 2 + 0) * N + n] / 2.0;
        jy += F[(s * 2 + 1) * N + n] / 2.0;
      }
      double r = rho[0 * N + n] + rho[1 * N + n];
      jx /= r;
      jy /= r;
    }
    u[0 * N + n] = jx;
    u[1 * N + n] = jy;
  }
}

void oracle_fields(const oracle_params *p, const unsigned char *mask,
                   const double *f, double *rho, double *rt, double *F,
                   double *u) {
  oracle_densities(p, mask, f, rho);
  if (p->bc == ORACLE_BC_VIRTUAL_AVG) {
    oracle_virtual_density(p, mask, rho, rt);
  } else {
    memset(rt, 0, sizeof(double) * 2 * (size_t)p->nx * p->ny);
  }
  oracle_forces(p, mask, rho, rt, F);
  oracle_velocity(p, mask, f, rho, F, u);
}

/* Right-hand side of Eq. 1 added to f: BGK relaxation towards Eq. 2 plus the
 * Guo source of Eq. 4, both evaluated with u^eq of Eq. 3. */
void oracle_collide(const oracle_params *p, const unsigned char *mask,
                    const double *f, const double *rho, const double *u,
                    const double *F, double *fpost) {
  long N = (long)p->nx * p->ny;
  for (int s = 0; s < 2; ++s)
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
      double feq[9], S[9];
      if (mask[n]) {
        for (int i = 0; i < 9; ++i) fpost[(s * 9 + i) * N + n] = 0.0;
        continue;
      }
      oracle_equilibrium(rho[s * N + n], u[n], u[N + n], feq);
      oracle_source(p->tau[s], u[n], u[N + n], F[(s * 2 + 0) * N + n],
                    F[(s * 2 + 1) * N + n], S);
      for (int i = 0; i < 9; ++i) {
        double fi = f[(s * 9 + i) * N + n];
        fpost[(s * 9 + i) * N + n] = fi - (fi - feq[i]) / p->tau[s] + S[i];
      }
    }
}

/* Left-hand side of Eq. 1 with halfway bounce-back: the population arriving
 * at fluid node x along c_i left x - c_i; when x - c_i is solid it is the
 * population that left x along -c_i, reflected. */
void oracle_stream(const oracle_params *p, const unsigned char *mask,
                   const double *fpost, double *f) {
  long N = (long)p->nx * p->ny;
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < 9; ++i) {
      int oi = opposite(i);
#pragma omp parallel for schedule(static)
      for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
          long n = (long)y * p->nx + x;
          double v = 0.0;
          if (!mask[n]) {
            long m = neighbour(p, x, y, -CX[i], -CY[i]);
            if (!phi(mask, m)) {
              v = fpost[(s * 9 + i) * N + m];
            } else {
              v = fpost[(s * 9 + oi) * N + n];
            }
          }
          f[(s * 9 + i) * N + n] = v;
        }
    }
}

int oracle_init(const oracle_params *p, const unsigned char *mask,
                const double *rhoA, const double *rhoB, const double *ux,
                const double *uy, double *f) {
  if (oracle_check(p, mask)) return 1;
  long N = (long)p->nx * p->ny;
  for (int s = 0; s < 2; ++s)
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
      double feq[9];
      const double *r = s ? rhoB : rhoA;
      double vx = ux ? ux[n] : 0.0, vy = uy ? uy[n] : 0.0;
      oracle_equilibrium(mask[n] ? 0.0 : r[n], vx, vy, feq);
      for (int i = 0; i < 9; ++i)
        f[(s * 9 + i) * N + n] = mask[n] ? 0.0 : feq[i];
    }
  return 0;
}

/* One time step of Eq. 1 per iteration, in the paper's order: densities,
 * virtual solid densities (improved scheme, every step, Sec. 3.2), forces,
 * common velocity, collision with source, streaming with bounce-back. */
int oracle_step(const oracle_params *p, const unsigned char *mask, double *f,
                int nsteps) {
  if (oracle_check(p, mask)) return 1;
  size_t N = (size_t)p->nx * p->ny;
  double *rho = (double *)malloc(sizeof(double) * 2 * N);
  double *rt = (double *)malloc(sizeof(double) * 2 * N);
  double *F = (double *)malloc(sizeof(double) * 4 * N);
  double *u = (double *)malloc(sizeof(double) * 2 * N);
  double *fpost = (double *)malloc(sizeof(double) * 18 * N);
  if (!rho || !rt || !F || !u || !fpost) {
    free(rho); free(rt); free(F); free(u); free(fpost);
    return 3;
  }
  for (int t = 0; t < nsteps; ++t) {
    oracle_fields(p, mask, f, rho, rt, F, u);
    oracle_collide(p, mask, f, rho, u, F, fpost);
    oracle_stream(p, mask, fpost, f);
  }
  free(rho); free(rt); free(F); free(u); free(fpost);
  return 0;
}

/* Total mass of each component over fluid nodes. */
void oracle_mass(const oracle_params *p, const unsigned char *mask,
                 const double *f, double *out) {
  long N = (long)p->nx * p->ny;
  for (int s = 0; s < 2; ++s) {
    double m = 0.0;
    for (long n = 0; n < N; ++n)
      if (!mask[n])
        for (int i = 0; i < 9; ++i) m += f[(s * 9 + i) * N + n];
    out[s] = m;
  }
}
