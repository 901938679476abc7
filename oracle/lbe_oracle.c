/*
 * Plain FP64 CPU oracle of one Lattice Boltzmann Electrokinetics (LBE) time
 * step with constant-potential (metallic) electrodes, after Asta, Palaia,
 * Trizac, Levesque and Rotenberg, "Lattice Boltzmann Electrokinetics
 * simulation of nanocapacitors" (arXiv:1907.04732).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only the tests, the
 * package's smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, table or header with the CUDA library.
 *
 * Units: lattice spacing = time step = 1, k_B T = e = 1.  phi is the reduced
 * potential beta*e*psi.  eps = 1/(4 pi l_B) plays the role of eps0*epsr.
 *
 * What one step computes, in this order (the paper lists the ingredients of
 * Sec. "Lattice Boltzmann Electrokinetics" but not their order):
 *   1. link fluxes j_k^i of Eq. LF2 from n_k(t), phi(t) (diffusion +
 *      migration), zero through fluid-solid links;
 *      n_k* = n_k(t) - sum_i j_k^i  (Eq. LF1 read with the A0 factor folded
 *      into d_k = D_k/A0 only, so that the effective diffusivity is D_k);
 *   2. force density on the solvent from the link excess fluxes
 *      g = j/d_k + (n' - n)/Delta_i,  F = (1/(2 A0)) sum_i c_i sum_k g;
 *   3. D3Q19 BGK collision (Eq. LBpop) with second-order equilibrium and
 *      Guo forcing, u = (sum_i f_i c_i + F/2)/rho, then streaming with
 *      halfway bounce-back at solid nodes;
 *   4. advection of n_k* by the velocity u(t) of step 3: the solute of a node
 *      moves with the node's displaced unit cell and is shared among the (up
 *      to 8) cells it overlaps, in proportion to the overlap volume; a share
 *      that would land on a solid node stays on the source node;
 *   5. Poisson solve (Eq. SOR's fixed point) with the modified Laplacian of
 *      Eq. DiscreteLaplacianModif on fluid nodes, solid nodes held at their
 *      electrode potential; warm-started from phi(t).
 * The induced charge (Eq. Qelec) is evaluated on demand from the current phi.
 *
 * The modified-Laplacian link factor is read as 1 + |chi(r+c_i) - chi(r)|:
 * identical to the printed 1 + chi(r+c_i) - chi(r) at fluid nodes, and the
 * doubling of every boundary link that the text of Sec. "Imposing conducting
 * boundary conditions" asks for at solid nodes (the printed sign would give
 * a zero factor there and hence Q = 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_Q 19
#define ORC_MAXS 4
#define ORC_MAXE 255

/* D3Q19 velocities: rest, 6 nearest neighbours, 12 next-nearest. */
static const int CV[ORC_Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

/* index of -c_i */
static int opposite(int i) {
  for (int j = 0; j < ORC_Q; ++j)
    if (CV[j][0] == -CV[i][0] && CV[j][1] == -CV[i][1] && CV[j][2] == -CV[i][2]) return j;
  return -1;
}

/* lattice weight w_i: 1/3, 1/18, 1/36 for |c|^2 = 0, 1, 2 */
static double weight(int i) {
  int c2 = CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
  if (c2 == 0) return 1.0 / 3.0;
  if (c2 == 1) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

/* Delta_i = |c_i| */
static double link_len(int i) {
  int c2 = CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
  return sqrt((double)c2);
}

static const double CS2 = 1.0 / 3.0;

typedef struct {
  int nx, ny, nz;
  int periodic[3];
  double tau;
  double bjerrum;
  int ns;
  double z[ORC_MAXS], D[ORC_MAXS], rho_bulk[ORC_MAXS];
  double e_app[3];
  double g_body[3];   /* external body force density on the solvent (0 unless set) */
  int node_rule;      /* 1: the first-order rule (solid nodes at psi, plain Laplacian) */
  int flow;
  double tol;
  int maxit;

  size_t N;
  int n_elec;
  uint8_t *id;        /* 0 fluid, e >= 1 electrode e */
  double psi[ORC_MAXE + 1];
  double *f;          /* f[i*N + r], populations after streaming (time t) */
  double *n;          /* n[k*N + r] */
  double *phi;        /* N */
  double *u;          /* u[a*N + r], velocity of the last collision */
  int last_iters;
  double last_res;
} orc;

static size_t idx(const orc *o, int x, int y, int zc) {
  return (size_t)x + (size_t)o->nx * ((size_t)y + (size_t)o->ny * (size_t)zc);
}

/* Neighbour of node (x,y,z) along integer offset (dx,dy,dz); -1 if it leaves a
 * non-periodic box. */
static long nbr_off(const orc *o, int x, int y, int zc, int dx, int dy, int dz) {
  int p[3] = {x + dx, y + dy, zc + dz};
  int L[3] = {o->nx, o->ny, o->nz};
  for (int a = 0; a < 3; ++a) {
    if (p[a] < 0 || p[a] >= L[a]) {
      if (!o->periodic[a]) return -1;
      p[a] = ((p[a] % L[a]) + L[a]) % L[a];
    }
  }
  return (long)idx(o, p[0], p[1], p[2]);
}

static void coords(const orc *o, size_t r, int *x, int *y, int *zc) {
  *x = (int)(r % (size_t)o->nx);
  *y = (int)((r / (size_t)o->nx) % (size_t)o->ny);
  *zc = (int)(r / ((size_t)o->nx * (size_t)o->ny));
}

static long nbr(const orc *o, size_t r, int i) {
  int x, y, zc;
  coords(o, r, &x, &y, &zc);
  return nbr_off(o, x, y, zc, CV[i][0], CV[i][1], CV[i][2]);
}

static int solid(const orc *o, long r) { return o->id[r] != 0; }

/* ------------------------------------------------------------------------ */
orc *orc_create(int nx, int ny, int nz, const int *periodic, double tau, double bjerrum,
                int ns, const double *zk, const double *Dk, const double *rho_bulk,
                const double *e_app, int flow, double tol, int maxit) {
  if (nx < 1 || ny < 1 || nz < 1 || ns < 1 || ns > ORC_MAXS) return NULL;
  orc *o = (orc *)calloc(1, sizeof(orc));
  o->nx = nx; o->ny = ny; o->nz = nz;
  for (int a = 0; a < 3; ++a) { o->periodic[a] = periodic[a]; o->e_app[a] = e_app[a]; }
  o->tau = tau; o->bjerrum = bjerrum; o->ns = ns;
  for (int k = 0; k < ns; ++k) { o->z[k] = zk[k]; o->D[k] = Dk[k]; o->rho_bulk[k] = rho_bulk[k]; }
  o->flow = flow; o->tol = tol; o->maxit = maxit;
  o->N = (size_t)nx * ny * nz;
  o->id = (uint8_t *)calloc(o->N, 1);
  o->f = (double *)calloc((size_t)ORC_Q * o->N, sizeof(double));
  o->n = (double *)calloc((size_t)ns * o->N, sizeof(double));
  o->phi = (double *)calloc(o->N, sizeof(double));
  o->u = (double *)calloc(3 * o->N, sizeof(double));
  return o;
}

void orc_destroy(orc *o) {
  if (!o) return;
  free(o->id); free(o->f); free(o->n); free(o->phi); free(o->u); free(o);
}

int orc_set_geometry(orc *o, const uint8_t *id, int n_elec) {
  if (n_elec < 0 || n_elec > ORC_MAXE) return -1;
  for (size_t r = 0; r < o->N; ++r) {
    if (id[r] > n_elec) return -1;
    o->id[r] = id[r];
  }
  o->n_elec = n_elec;
  /* every fluid node must keep all its D3Q19 and cube-corner neighbours
   * inside the box: a non-periodic face has to be solid */
  for (size_t r = 0; r < o->N; ++r) {
    if (o->id[r]) continue;
    int x, y, zc;
    coords(o, r, &x, &y, &zc);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx)
          if (nbr_off(o, x, y, zc, dx, dy, dz) < 0) return -2;
  }
  return 0;
}

int orc_set_voltage(orc *o, const double *psi) {
  o->psi[0] = 0.0;
  for (int e = 1; e <= o->n_elec; ++e) o->psi[e] = psi[e - 1];
  for (size_t r = 0; r < o->N; ++r)
    if (o->id[r]) o->phi[r] = o->psi[o->id[r]];
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Link factor of the Laplacian: 1 + |chi(r+c_i) - chi(r)| in Eq.
 * DiscreteLaplacianModif; 1 on every link under the first-order rule that
 * the paper describes before it (Eq. DiscreteLaplacian, solid nodes simply
 * held at their potential, which puts the interface on the solid node). */
static double link_factor(const orc *o, long r, long r2) {
  if (o->node_rule) return 1.0;
  return 1.0 + fabs((double)solid(o, r2) - (double)solid(o, r));
}

/* Eq. DiscreteLaplacianModif: (2/c_s^2) sum_i w_i [phi(r+c_i) - phi(r)] *
 * [1 + |chi(r+c_i) - chi(r)|], evaluated at any node r.  Links that leave a
 * non-periodic box are skipped (they only exist at solid faces and join
 * nodes of one electrode).                                                 */
static double laplacian_at(const orc *o, const double *phi, size_t r) {
  double s = 0.0;
  for (int i = 1; i < ORC_Q; ++i) {
    long r2 = nbr(o, r, i);
    if (r2 < 0) continue;
    double factor = link_factor(o, (long)r, r2);
    s += (2.0 / CS2) * weight(i) * (phi[r2] - phi[r]) * factor;
  }
  return s;
}

void orc_laplacian(const orc *o, const double *phi, double *out) {
  for (size_t r = 0; r < o->N; ++r) out[r] = laplacian_at(o, phi, r);
}

/* rho_el = sum_k z_k n_k (Eq. Poisson), per node */
static void charge_density(const orc *o, const double *n, double *rho_el) {
  for (size_t r = 0; r < o->N; ++r) {
    double q = 0.0;
    for (int k = 0; k < o->ns; ++k) q += o->z[k] * n[(size_t)k * o->N + r];
    rho_el[r] = q;
  }
}

/* Diagonal of the operator phi -> -laplacian on the fluid unknowns (links to
 * the node itself, which exist only in boxes one node wide, cancel). */
static double diag_at(const orc *o, size_t r) {
  double d = 0.0;
  for (int i = 1; i < ORC_Q; ++i) {
    long r2 = nbr(o, r, i);
    if (r2 < 0 || (size_t)r2 == r) continue;
    double factor = link_factor(o, (long)r, r2);
    d += (2.0 / CS2) * weight(i) * factor;
  }
  return d;
}

/* Poisson solve: find phi on fluid nodes with
 *   laplacian(phi)(r) + 4 pi l_B rho_el(r) = 0,
 * solid nodes fixed at their electrode potential.  The paper iterates Eq. SOR
 * and takes the converged potential; the converged potential is what this
 * computes, by Jacobi-preconditioned conjugate gradients on the symmetric
 * positive (semi-)definite system.  Stops when max_r |res(r)|/diag(r) <= tol.
 * Returns the number of iterations, or -1 if maxit was reached. */
static int poisson_solve(orc *o, const double *rho_el) {
  size_t N = o->N;
  double four_pi_lb = 4.0 * M_PI * o->bjerrum;
  double *res = (double *)calloc(N, sizeof(double));
  double *zv = (double *)calloc(N, sizeof(double));
  double *p = (double *)calloc(N, sizeof(double));
  double *q = (double *)calloc(N, sizeof(double));
  double *dg = (double *)calloc(N, sizeof(double));
  double *tmp = (double *)calloc(N, sizeof(double));
  for (size_t r = 0; r < N; ++r)
    if (!o->id[r]) dg[r] = diag_at(o, r);

  /* residual b - A phi = laplacian(phi) + 4 pi l_B rho_el on fluid nodes */
#pragma omp parallel for schedule(static)
  for (size_t r = 0; r < N; ++r)
    res[r] = o->id[r] ? 0.0 : laplacian_at(o, o->phi, r) + four_pi_lb * rho_el[r];

  int it = 0, ok = 0;
  double rz = 0.0;
  for (size_t r = 0; r < N; ++r)
    if (!o->id[r]) { zv[r] = res[r] / dg[r]; p[r] = zv[r]; rz += res[r] * zv[r]; }
  for (it = 0; it <= o->maxit; ++it) {
    double rmax = 0.0;
    for (size_t r = 0; r < N; ++r)
      if (!o->id[r]) { double a = fabs(res[r]) / dg[r]; if (a > rmax) rmax = a; }
    o->last_res = rmax;
    if (rmax <= o->tol) { ok = 1; break; }
    if (it == o->maxit) break;
    /* q = A p, with A = -laplacian restricted to fluid unknowns (p = 0 on
     * solid nodes) */
    for (size_t r = 0; r < N; ++r) tmp[r] = o->id[r] ? 0.0 : p[r];
#pragma omp parallel for schedule(static)
    for (size_t r = 0; r < N; ++r) q[r] = o->id[r] ? 0.0 : -laplacian_at(o, tmp, r);
    double pq = 0.0;
    for (size_t r = 0; r < N; ++r) pq += p[r] * q[r];
    if (pq <= 0.0) { ok = (rmax <= o->tol); break; }
    double alpha = rz / pq;
    for (size_t r = 0; r < N; ++r)
      if (!o->id[r]) { o->phi[r] += alpha * p[r]; res[r] -= alpha * q[r]; }
    double rz_new = 0.0;
    for (size_t r = 0; r < N; ++r)
      if (!o->id[r]) { zv[r] = res[r] / dg[r]; rz_new += res[r] * zv[r]; }
    double beta = rz_new / rz;
    rz = rz_new;
    for (size_t r = 0; r < N; ++r)
      if (!o->id[r]) p[r] = zv[r] + beta * p[r];
    /* refresh the true residual now and then against drift */
    if ((it + 1) % 50 == 0)
#pragma omp parallel for schedule(static)
      for (size_t r = 0; r < N; ++r)
        res[r] = o->id[r] ? 0.0 : laplacian_at(o, o->phi, r) + four_pi_lb * rho_el[r];
  }
  o->last_iters = it;
  free(res); free(zv); free(p); free(q); free(dg); free(tmp);
  return ok ? it : -1;
}

int orc_poisson(orc *o, const double *rho_el) { return poisson_solve(o, rho_el); }

/* ---------------------------------------------------------------------- */
/* Eq. LF2 for one link and one species, in the relative form obtained by
 * multiplying numerator and denominator by exp(-beta mu(r)):
 *   j = -d/Delta * (1/2)(1 + e^{-dmu}) (n' e^{dmu} - n),
 * dmu = beta(mu(r+c_i) - mu(r)) = z (phi' - phi - E_app . c_i).
 * (Identical to the printed form; the relative form keeps an applied field
 * well defined in a periodic box.)                                        */
double orc_link_flux(double d, double delta_len, double zk, double phi0, double phi1,
                     double e_dot_c, double n0, double n1) {
  double dmu = zk * (phi1 - phi0 - e_dot_c);
  double avg = 0.5 * (1.0 + exp(-dmu));
  return -d * avg * (n1 * exp(dmu) - n0) / delta_len;
}

static const double A0 = 1.0 + 2.0 * 1.4142135623730951; /* 1 + 2 sqrt(2) */

/* Steps 1-2: n* and the solvent force density F (3 per node). */
static void ion_fluxes(const orc *o, double *nstar, double *F) {
  size_t N = o->N;
  memcpy(nstar, o->n, sizeof(double) * (size_t)o->ns * N);
  memset(F, 0, sizeof(double) * 3 * N);
#pragma omp parallel for schedule(static)
  for (size_t r = 0; r < N; ++r) {
    if (o->id[r]) continue;
    double force[3] = {0, 0, 0};
    for (int i = 1; i < ORC_Q; ++i) {
      long r2 = nbr(o, r, i);
      if (r2 < 0 || o->id[r2]) continue; /* no flux through fluid-solid links */
      double e_dot_c = o->e_app[0] * CV[i][0] + o->e_app[1] * CV[i][1] + o->e_app[2] * CV[i][2];
      double dl = link_len(i);
      double g = 0.0;
      for (int k = 0; k < o->ns; ++k) {
        double d = o->D[k] / A0;
        double n0 = o->n[(size_t)k * N + r], n1 = o->n[(size_t)k * N + (size_t)r2];
        double j = orc_link_flux(d, dl, o->z[k], o->phi[r], o->phi[r2], e_dot_c, n0, n1);
        nstar[(size_t)k * N + r] -= j;
        g += j / d + (n1 - n0) / dl;
      }
      for (int a = 0; a < 3; ++a) force[a] += CV[i][a] * g;
    }
    for (int a = 0; a < 3; ++a) F[(size_t)a * N + r] = force[a] / (2.0 * A0) + o->g_body[a];
  }
}

/* second-order equilibrium w_i rho [1 + c.u/cs2 + (c.u)^2/(2 cs2^2) - u^2/(2 cs2)] */
static double feq(int i, double rho, const double *u) {
  double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return weight(i) * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Guo forcing term (1 - 1/(2 tau)) w_i [ (c_i - u)/cs2 + (c_i.u) c_i / cs2^2 ] . F */
static double guo(int i, double tau, const double *u, const double *Fv) {
  double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
  double s = 0.0;
  for (int a = 0; a < 3; ++a)
    s += ((CV[i][a] - u[a]) / CS2 + cu * CV[i][a] / (CS2 * CS2)) * Fv[a];
  return (1.0 - 1.0 / (2.0 * tau)) * weight(i) * s;
}

static void moments(const orc *o, size_t r, const double *Fv, double *rho, double *u) {
  size_t N = o->N;
  double m[3] = {0, 0, 0}, s = 0.0;
  for (int i = 0; i < ORC_Q; ++i) {
    double fi = o->f[(size_t)i * N + r];
    s += fi;
    for (int a = 0; a < 3; ++a) m[a] += fi * CV[i][a];
  }
  *rho = s;
  for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * Fv[a]) / s;
}

/* Step 3: Eq. LBpop with BGK + Guo forcing, then streaming with halfway
 * bounce-back. */
static void lb_collide_stream(orc *o, const double *F) {
  size_t N = o->N;
  double *fnew = (double *)calloc((size_t)ORC_Q * N, sizeof(double));
  /* each (i, destination) slot has exactly one writer, so nodes are
   * independent */
#pragma omp parallel for schedule(static)
  for (size_t r = 0; r < N; ++r) {
    if (o->id[r]) continue;
    double fpost[ORC_Q];
    double Fv[3] = {F[r], F[N + r], F[2 * N + r]};
    double rho, u[3];
    moments(o, r, Fv, &rho, u);
    for (int a = 0; a < 3; ++a) o->u[(size_t)a * N + r] = u[a];
    for (int i = 0; i < ORC_Q; ++i) {
      double fi = o->f[(size_t)i * N + r];
      fpost[i] = fi - (fi - feq(i, rho, u)) / o->tau + guo(i, o->tau, u, Fv);
    }
    for (int i = 0; i < ORC_Q; ++i) {
      long r2 = i == 0 ? (long)r : nbr(o, r, i);
      if (r2 >= 0 && !o->id[r2])
        fnew[(size_t)i * N + (size_t)r2] = fpost[i];
      else
        fnew[(size_t)opposite(i) * N + r] = fpost[i]; /* bounce back */
    }
  }
  memcpy(o->f, fnew, sizeof(double) * ORC_Q * N);
  free(fnew);
}

/* overlap length of a unit interval displaced by u with the cell at offset s
 * (s in {-1,0,1}), |u| < 1 */
static double overlap1(int s, double u) {
  if (s == 0) return 1.0 - fabs(u);
  if (s == 1) return u > 0.0 ? u : 0.0;
  return u < 0.0 ? -u : 0.0;
}

/* Step 4: advection of nstar by the velocity field u (cell-overlap rule). */
void orc_advect(const orc *o, const double *nin, const double *u, double *nout) {
  size_t N = o->N;
  memset(nout, 0, sizeof(double) * (size_t)o->ns * N);
  for (size_t r = 0; r < N; ++r) {
    if (o->id[r]) continue;
    int x, y, zc;
    coords(o, r, &x, &y, &zc);
    double uv[3] = {u[r], u[N + r], u[2 * N + r]};
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          double w = overlap1(dx, uv[0]) * overlap1(dy, uv[1]) * overlap1(dz, uv[2]);
          if (w == 0.0) continue;
          long r2 = nbr_off(o, x, y, zc, dx, dy, dz);
          if (r2 < 0 || o->id[r2]) r2 = (long)r; /* a share bound for a solid node stays */
          for (int k = 0; k < o->ns; ++k)
            nout[(size_t)k * N + (size_t)r2] += w * nin[(size_t)k * N + r];
        }
  }
}

/* ---------------------------------------------------------------------- */
/* Initial condition (Sec. "Potential and concentration profiles"): uncharged
 * capacitor with uniform bulk concentrations on fluid nodes, fluid at rest
 * with unit density, potential = Laplace solution for the applied voltage. */
int orc_init(orc *o) {
  size_t N = o->N;
  for (size_t r = 0; r < N; ++r) {
    for (int k = 0; k < o->ns; ++k) o->n[(size_t)k * N + r] = o->id[r] ? 0.0 : o->rho_bulk[k];
    for (int i = 0; i < ORC_Q; ++i) o->f[(size_t)i * N + r] = o->id[r] ? 0.0 : weight(i);
    for (int a = 0; a < 3; ++a) o->u[(size_t)a * N + r] = 0.0;
    o->phi[r] = o->id[r] ? o->psi[o->id[r]] : 0.0;
  }
  double *rho_el = (double *)malloc(sizeof(double) * N);
  charge_density(o, o->n, rho_el);
  int it = poisson_solve(o, rho_el);
  free(rho_el);
  return it < 0 ? -3 : 0;
}

int orc_step(orc *o, int nsteps) {
  size_t N = o->N;
  double *nstar = (double *)malloc(sizeof(double) * (size_t)o->ns * N);
  double *F = (double *)malloc(sizeof(double) * 3 * N);
  double *rho_el = (double *)malloc(sizeof(double) * N);
  int rc = 0;
  for (int s = 0; s < nsteps; ++s) {
    ion_fluxes(o, nstar, F);
    if (o->flow) {
      lb_collide_stream(o, F);
      orc_advect(o, nstar, o->u, o->n);
    } else {
      memcpy(o->n, nstar, sizeof(double) * (size_t)o->ns * N);
    }
    charge_density(o, o->n, rho_el);
    if (poisson_solve(o, rho_el) < 0) { rc = -3; break; }
  }
  free(nstar); free(F); free(rho_el);
  return rc;
}

/* Eq. Qelec: Q_e = -(1/(4 pi l_B)) sum_{r in e} laplacian(phi)(r), with the
 * modified Laplacian (the plain one under the first-order rule); only links
 * from electrode e to fluid nodes are taken (links between two electrodes
 * carry no induced charge of either). */
int orc_charge(const orc *o, double *q) {
  double eps = 1.0 / (4.0 * M_PI * o->bjerrum);
  for (int e = 0; e < o->n_elec; ++e) q[e] = 0.0;
  for (size_t r = 0; r < o->N; ++r) {
    int e = o->id[r];
    if (!e) continue;
    double s = 0.0;
    for (int i = 1; i < ORC_Q; ++i) {
      long r2 = nbr(o, r, i);
      if (r2 < 0 || o->id[r2]) continue;
      s += (2.0 / CS2) * weight(i) * (o->phi[r2] - o->phi[r]) * link_factor(o, (long)r, r2);
    }
    q[e - 1] += -eps * s;
  }
  return 0;
}

/* which: 0 phi (N), 1 n (ns*N), 2 rho (N), 3 u (3N, velocity at the current
 * time: (sum f c + F/2)/rho with F from the current n and phi), 4 f (19N) */
int orc_fields(orc *o, int which, double *out) {
  size_t N = o->N;
  if (which == 0) { memcpy(out, o->phi, sizeof(double) * N); return 0; }
  if (which == 1) { memcpy(out, o->n, sizeof(double) * (size_t)o->ns * N); return 0; }
  if (which == 4) { memcpy(out, o->f, sizeof(double) * ORC_Q * N); return 0; }
  if (which == 2 || which == 3) {
    double *nstar = (double *)malloc(sizeof(double) * (size_t)o->ns * N);
    double *F = (double *)malloc(sizeof(double) * 3 * N);
    ion_fluxes(o, nstar, F);
    for (size_t r = 0; r < N; ++r) {
      double rho = 0.0, u[3] = {0, 0, 0};
      if (!o->id[r]) {
        double Fv[3] = {F[r], F[N + r], F[2 * N + r]};
        moments(o, r, Fv, &rho, u);
        if (!o->flow) u[0] = u[1] = u[2] = 0.0;
      }
      if (which == 2) out[r] = rho;
      else for (int a = 0; a < 3; ++a) out[(size_t)a * N + r] = u[a];
    }
    free(nstar); free(F);
    return 0;
  }
  return -1;
}

/* Boundary rule of the Poisson solve: 0 (default) the paper's rule, Eq.
 * DiscreteLaplacianModif; 1 the first-order rule it improves on (plain Eq.
 * DiscreteLaplacian with the solid nodes held at their potential).  Set it
 * before orc_init. */
int orc_set_boundary_rule(orc *o, int node_rule) {
  o->node_rule = node_rule ? 1 : 0;
  return 0;
}

/* A uniform external body force density g on the solvent, added on every
 * fluid node to the ion force of step 2 (the force term of Eq. LBpop does not
 * care where the force comes from).  Zero unless set; it lets the pins drive
 * the lattice Boltzmann part alone (Poiseuille flow, momentum budget). */
int orc_set_body_force(orc *o, const double *g) {
  for (int a = 0; a < 3; ++a) o->g_body[a] = g[a];
  return 0;
}

/* Overwrite the dynamic state (any pointer may be NULL to keep it). */
int orc_set_state(orc *o, const double *f, const double *n, const double *phi) {
  size_t N = o->N;
  if (f) memcpy(o->f, f, sizeof(double) * ORC_Q * N);
  if (n) memcpy(o->n, n, sizeof(double) * (size_t)o->ns * N);
  if (phi) memcpy(o->phi, phi, sizeof(double) * N);
  return 0;
}

/* Solvent force density of step 2 for the current state (3N). */
int orc_force(const orc *o, double *F) {
  double *nstar = (double *)malloc(sizeof(double) * (size_t)o->ns * o->N);
  ion_fluxes(o, nstar, F);
  free(nstar);
  return 0;
}

int orc_last_iters(const orc *o) { return o->last_iters; }
double orc_last_res(const orc *o) { return o->last_res; }
