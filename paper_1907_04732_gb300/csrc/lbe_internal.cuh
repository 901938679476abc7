// Internal declarations of the GB300 LBE library: lattice geometry helpers,
// the D3Q19 velocity set, the handle and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lbe.h"

namespace lbe {

// D3Q19 velocity set: 0 = rest; 1..9 one half of the moving velocities and
// 10..18 their opposites (opp(i) = i +- 9).  Weights 1/3, 1/18, 1/36 and
// c_s^2 = 1/3 (Sec. "Lattice Boltzmann Electrokinetics").
constexpr int kQ = 19;
__host__ __device__ constexpr int cx_of(int i) {
  constexpr int t[kQ] = {0, 1, 0, 0, 1, 1, 1, 1, 0, 0, -1, 0, 0, -1, -1, -1, -1, 0, 0};
  return t[i];
}
__host__ __device__ constexpr int cy_of(int i) {
  constexpr int t[kQ] = {0, 0, 1, 0, 1, -1, 0, 0, 1, 1, 0, -1, 0, -1, 1, 0, 0, -1, -1};
  return t[i];
}
__host__ __device__ constexpr int cz_of(int i) {
  constexpr int t[kQ] = {0, 0, 0, 1, 0, 0, 1, -1, 1, -1, 0, 0, -1, 0, 0, -1, 1, -1, 1};
  return t[i];
}
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : (i <= 9 ? i + 9 : i - 9); }
__host__ __device__ constexpr int c2_of(int i) {
  return cx_of(i) * cx_of(i) + cy_of(i) * cy_of(i) + cz_of(i) * cz_of(i);
}
__host__ __device__ constexpr double w_of(int i) {
  return c2_of(i) == 0 ? 1.0 / 3.0 : (c2_of(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}
// (2/c_s^2) w_i: the Laplacian link coefficient of Eq. DiscreteLaplacian
__host__ __device__ constexpr double lapc_of(int i) { return c2_of(i) == 1 ? 1.0 / 3.0 : 1.0 / 6.0; }
// 1/|c_i|
__host__ __device__ constexpr double invlen_of(int i) {
  return c2_of(i) == 1 ? 1.0 : 0.70710678118654752440;
}

// Per-node link mask: bit (i-1), i = 1..18, set when the D3Q19 neighbour
// r + c_i is inside the box and fluid; bits 18..25 the same for the eight
// cube corners (+-1,+-1,+-1), corner index 18 + (sx>0) + 2(sy>0) + 4(sz>0);
// bit 31 set when r itself is fluid.
constexpr uint32_t kFluidBit = 1u << 31;
constexpr uint32_t kLinkBits = 0x3FFFFu;  // the 18 link bits
__host__ __device__ constexpr int corner_bit(int sx, int sy, int sz) {
  return 18 + (sx > 0) + 2 * (sy > 0) + 4 * (sz > 0);
}

struct Geo {
  int nx, ny, nz;
  int px, py, pz;  // periodic flags
  long long N;
};

__host__ __device__ inline void coords(const Geo &g, long long r, int &x, int &y, int &z) {
  x = (int)(r % g.nx);
  long long t = r / g.nx;
  y = (int)(t % g.ny);
  z = (int)(t / g.ny);
}

// Neighbour index at integer offset (dx,dy,dz) in {-1,0,1}^3, -1 when it
// leaves a non-periodic box.
__host__ __device__ inline long long nbr(const Geo &g, int x, int y, int z, int dx, int dy, int dz) {
  int X = x + dx, Y = y + dy, Z = z + dz;
  if (X < 0 || X >= g.nx) { if (!g.px) return -1; X = X < 0 ? X + g.nx : X - g.nx; }
  if (Y < 0 || Y >= g.ny) { if (!g.py) return -1; Y = Y < 0 ? Y + g.ny : Y - g.ny; }
  if (Z < 0 || Z >= g.nz) { if (!g.pz) return -1; Z = Z < 0 ? Z + g.nz : Z - g.nz; }
  return (long long)X + (long long)g.nx * ((long long)Y + (long long)g.ny * Z);
}

// 3-D launch geometry: 256-thread blocks tiled over (x, y, z), x fastest, so
// that node coordinates come from the thread indices (no divisions).  Each
// thread visits zpt z-planes (zpt > 1 bounds the block count of kernels that
// write one reduction partial per block).
struct Launch {
  dim3 grid, block;
  int zpt;
  long long nblk() const { return (long long)grid.x * grid.y * grid.z; }
};

inline int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

inline Launch make_launch(const Geo &g, long long max_blocks = 0) {
  const int bx = pow2_at_least(g.nx) < 256 ? pow2_at_least(g.nx) : 256;
  int by = pow2_at_least(g.ny) < 256 / bx ? pow2_at_least(g.ny) : 256 / bx;
  int bz = 256 / (bx * by);
  if (bz > 64) {  // blockDim.z <= 64: widen the block along y instead
    bz = 64;
    by = 256 / (bx * bz);
  }
  Launch L;
  L.block = dim3(bx, by, bz);
  const long long gx = (g.nx + bx - 1) / bx, gy = (g.ny + by - 1) / by, gz0 = (g.nz + bz - 1) / bz;
  L.zpt = 1;
  if (max_blocks > 0 && gx * gy * gz0 > max_blocks)
    L.zpt = (int)((gx * gy * gz0 + max_blocks - 1) / max_blocks);
  L.grid = dim3((unsigned)gx, (unsigned)gy, (unsigned)((gz0 + L.zpt - 1) / L.zpt));
  return L;
}

// coordinates of this thread's node on z-pass kz; false when outside the box
__device__ __forceinline__ bool node_of(const Geo &g, int zpt, int kz, int &x, int &y, int &z, long long &r) {
  x = blockIdx.x * blockDim.x + threadIdx.x;
  y = blockIdx.y * blockDim.y + threadIdx.y;
  z = (blockIdx.z * zpt + kz) * blockDim.z + threadIdx.z;
  if (x >= g.nx || y >= g.ny || z >= g.nz) return false;
  r = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
  return true;
}

// Neighbour offsets of a node, periodic wrap included: the index of the
// neighbour at (dx,dy,dz) in {-1,0,1}^3 is r + off(dx,dy,dz).  32-bit: the
// library limits a lattice to fewer than 2^31 nodes.  On a non-periodic face
// the wrapped offset is never used by fluid nodes (those faces are solid).
// true when every link of a node joins a fluid node other than itself
// (most nodes of a lattice): the Laplacian's link weights are then
// constants, with no per-link tests
__device__ __forceinline__ bool all_links(uint32_t m, uint32_t selfmask) {
  return (m & kLinkBits) == kLinkBits && !(selfmask & kLinkBits);
}

struct Offs {
  int xm, xp, ym, yp, zm, zp;
  __device__ __forceinline__ int at(int dx, int dy, int dz) const {
    return (dx < 0 ? xm : (dx > 0 ? xp : 0)) + (dy < 0 ? ym : (dy > 0 ? yp : 0)) + (dz < 0 ? zm : (dz > 0 ? zp : 0));
  }
};
__device__ __forceinline__ Offs offsets_of(const Geo &g, int x, int y, int z) {
  const int sy = g.nx, sz = g.nx * g.ny;
  Offs o;
  o.xm = x == 0 ? g.nx - 1 : -1;
  o.xp = x == g.nx - 1 ? 1 - g.nx : 1;
  o.ym = y == 0 ? (g.ny - 1) * sy : -sy;
  o.yp = y == g.ny - 1 ? (1 - g.ny) * sy : sy;
  o.zm = z == 0 ? (g.nz - 1) * sz : -sz;
  o.zp = z == g.nz - 1 ? (1 - g.nz) * sz : sz;
  return o;
}

// A term of a max |residual| stopping test with NaN read as +infinity: fmax
// drops NaN operands, so a NaN residual would otherwise vanish from the test.
__device__ __forceinline__ float finite_or_inf(float v) { return v == v ? v : __int_as_float(0x7f800000); }
__device__ __forceinline__ double finite_or_inf(double v) { return v == v ? v : __longlong_as_double(0x7ff0000000000000LL); }

__device__ __forceinline__ int flat_tid() {
  return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}
__device__ __forceinline__ long long flat_bid() {
  return blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
}

// Physical constants of one lattice, passed by value to kernels.
struct Phys {
  int ns;
  double z[LBE_MAX_SPECIES];
  double d[LBE_MAX_SPECIES];      // D_k / A0
  double inv_d[LBE_MAX_SPECIES];  // A0 / D_k
  double e_dot_c[kQ];             // E_app . c_i
  double tau, omega;              // omega = 1/tau
  double guo;                     // 1 - 1/(2 tau)
  double four_pi_lb;
  double eps;                     // 1/(4 pi l_B)
  double inv_2a0;                 // 1/(2 A0)
  uint32_t selfmask;              // links that join a node to itself (| kPlainLaplacian)
  double solid_factor;            // factor of the links to solid: 2 (Eq. DiscreteLaplacianModif) or 1
};
// Flag kept in Phys::selfmask (above the 18 link bits) by the first-order
// boundary rule: the Poisson stencils then leave the links to solid
// undoubled (LBE_RULE_NODE; FP64 form only).
constexpr uint32_t kPlainLaplacian = 1u << 30;

// Constants of the FP32 form.  Solute amounts are int64 fixed point:
// n_k = rho_k^bulk + s_k q_k with s_k = rho_k^bulk 2^-kFixBits (solid nodes
// hold q = -2^kFixBits, i.e. n = 0).  The unit is fine enough that rounding
// each link flux to it leaves no measurable bias even where the fluxes are
// smooth in space and time.
constexpr int kFixBits = 40;
struct P32 {
  int ns;
  int zi[LBE_MAX_SPECIES];
  float zf[LBE_MAX_SPECIES];
  float rb[LBE_MAX_SPECIES], s[LBE_MAX_SPECIES];
  double rbd[LBE_MAX_SPECIES], sd[LBE_MAX_SPECIES];
  float kq1[LBE_MAX_SPECIES], kq2[LBE_MAX_SPECIES];  // -d_k/(2|c| s_k), |c| = 1, sqrt 2
  float ec[kQ];                                      // E_app . c_i, ec[opp] = -ec
  float omega, guo, inv_2a0;
  int salt11;  // two species, z = +1 and -1, equal bulk concentrations
};

// Deterministic block reductions (fixed tree order).
constexpr int kBlock = 256;

// Control block of the Poisson solves (device memory; see poisson.cu).
struct PoissonCtl {
  int outer_done, inner_done, rounds, status, sticky_status, arrive;
  long long solve_iters, total_iters, total_rounds, solves, max_solve_iters;
  double res, res0, alpha, beta, gamma;
  double ref;  // linear solves: max |rhs|/diag, the scale of the relative test
};

struct PoissonWork {
  void *vec = nullptr;        // CG vectors r, u, w, x, p, s ([6][N], FP32 or FP64)
  double *partial = nullptr;  // block partials [3][nblk]
  PoissonCtl *ctl = nullptr;  // device
  PoissonCtl *ctl_host = nullptr;  // pinned
  Launch L{};                 // launch of the CG kernels (<= kMaxPartials blocks)
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  const void *exec_key[2] = {nullptr, nullptr};
  cudaGraphExec_t exec_lin = nullptr;  // linear solve A x = rhs (adjoint)
  const void *lin_key[3] = {nullptr, nullptr, nullptr};
  bool graph_ok = false;
  double *phi_prev = nullptr;  // [kHist][N]: phi of the previous kHist steps (warm start;
                               // the FP32 form keeps fixed-point values, int64, in it)
  int history = 0;             // how many of them hold a solution (0..kHist)
};
constexpr int kMaxPartials = 2048;
// Order of the warm start's extrapolation in time = the number of earlier
// solutions kept (fp32::extrapolate_node).
#ifndef LBE_EXTRAP_ORDER
#define LBE_EXTRAP_ORDER 3
#endif
constexpr int kHist = LBE_EXTRAP_ORDER;
// The FP32 form's potential in fixed point: phi = phifx * 2^-kPhiFixBits.
// The unit 2^-48 (3.6e-15) lies far below the solve tolerance; |phi| below
// kPhiMax keeps every integer sum of the solve (18 weighted link
// differences, the cubic warm start) far from 2^63.
constexpr int kPhiFixBits = 48;
constexpr double kPhiMax = 100.0;
static_assert(kHist >= 1 && kHist <= 3, "extrapolation order 1..3");
// Launch size of the solve's lattice kernels: each thread handles zpt nodes
// along z so that a kernel has at most this many blocks.  On this GPU a
// dependent kernel costs about 0.6 ns per block to schedule (2.4 us for 4096
// empty blocks of 256 threads, 0.4 us for one block), which the short
// kernels of the solve pay dozens of times per step.
#ifndef LBE_SOLVE_BLOCKS
#define LBE_SOLVE_BLOCKS 1024
#endif
constexpr int kSolveBlocks = LBE_SOLVE_BLOCKS;

// Multigrid hierarchy of the FP32 Poisson preconditioner (mg.cu); level 0 is
// the lattice itself.
constexpr int kMaxLevels = 10;
struct MGLevel {
  int nx = 0, ny = 0, nz = 0, sx = 0, sy = 0, sz = 0;
  long long N = 0;
  float *A = nullptr;  // 27-point Galerkin operator [27][N]
  float *r = nullptr, *e = nullptr, *t = nullptr;
  float *z = nullptr;  // pre-smoothed iterate omega r/diag
};
struct MGWork {
  MGLevel lv[kMaxLevels];
  int nlev = 0;        // 0: no hierarchy (Jacobi preconditioning)
  float *t0 = nullptr;  // fine-level scratch
  float *cinv = nullptr;  // inverse of the coarsest operator [N][N] (null: Jacobi sweeps)
};

struct AdjWork;  // adjoint.cu

}  // namespace lbe

struct lbe_handle {
  lbe_params prm{};
  lbe::Geo geo{};
  lbe::Phys phys{};
  lbe::P32 p32{};
  cudaStream_t stream = nullptr;
  bool owns_stream = false;           // stream created by the library
  int n_elec = 0;
  bool have_geometry = false;
  bool initialised = false;
  double psi[LBE_MAX_ELECTRODES] = {};
  std::string err;
  lbe_stats stats{};

  // device state
  uint8_t *id = nullptr;
  uint32_t *mask = nullptr;
  double *f[2] = {nullptr, nullptr};  // post-collision populations, [i][r]
  int cur = 0;                        // f[cur] holds the latest populations
  double *n = nullptr;                // [k][r]
  double *nstar = nullptr;            // [k][r]
  double *phi = nullptr;
  double *u = nullptr;                // [a][r], velocity of the last collision
  double *qpart = nullptr;            // charge partials [nblk][n_elec]
  double *qout = nullptr;             // [n_elec]
  double *qhost = nullptr;            // pinned
  double *psi_dev = nullptr;          // [LBE_MAX_ELECTRODES+1], index = electrode id
  int qblk = 0;
  lbe::PoissonWork pw;
  lbe::MGWork mg;

  // FP32 form state
  float *f32[2] = {nullptr, nullptr};  // population deviations f_i - w_i: f32[0], updated in place
  bool aa_odd = false;                 // the next step is an odd one of the AA pattern (fp32::PopLayout)
  int64_t *q = nullptr;                // fixed-point solute amounts [k][r]
  int64_t *qstar = nullptr;
  int64_t *phifx = nullptr;            // the potential in fixed point (kPhiFixBits), the master copy
  float *phi32 = nullptr;              // nearest float of phifx (the sweep's link records)
  bool phi64_stale = false;            // phi (FP64, the API's copy) lags phifx
  float4 *u32 = nullptr;               // velocity of the last collision (fp32::octant_code records)
  int *flag = nullptr;                 // device error flags (fixed-point range)
  float4 *lf = nullptr;                // 1:1 salt link records, one per node (fp32::link_record)
  float *pw32 = nullptr;               // FP32 Poisson work: res, p, q, e [4][N]

  // profiling (lbe_profile_begin/end): events [sweep start, sweep end,
  // advect end, poisson end] per step
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  long long launches = 0;     // kernels launched since profile_begin
  long long prof_iters = 0, prof_solves = 0, prof_steps = 0;

  // reverse-mode derivative (lbe_adjoint_*): checkpoints and work arrays;
  // gen counts the calls that change the state, so a backward pass can tell
  // whether the state it differentiates is still the forward pass's
  lbe::AdjWork *adj = nullptr;
  long long gen = 0;
};

namespace lbe {
// kernels_fp64.cu
cudaError_t launch_build_mask(const Geo &g, const uint8_t *id, uint32_t *mask, cudaStream_t s);
cudaError_t launch_init_state(lbe_handle *h);
cudaError_t launch_init_phi(lbe_handle *h);
cudaError_t launch_set_solid_phi(lbe_handle *h);
cudaError_t launch_sweep(lbe_handle *h);
cudaError_t launch_advect(lbe_handle *h);
cudaError_t launch_moments(lbe_handle *h, double *rho_out, double *u_out);
cudaError_t launch_gather_f(lbe_handle *h, double *out);
cudaError_t launch_charge(lbe_handle *h);
cudaError_t launch_charge_node(lbe_handle *h, double *out);
// kernels_fp32.cu
cudaError_t launch_init32(lbe_handle *h);
cudaError_t launch_sweep32(lbe_handle *h);
// extrapolate: also the warm start of the next solve (as k_extrapolate, with
// the current history), the advection not reading the potential
cudaError_t launch_advect32(lbe_handle *h, bool extrapolate = false);
cudaError_t launch_n_to_double(lbe_handle *h, double *out);
cudaError_t launch_n_from_double(lbe_handle *h, const double *n);
cudaError_t launch_moments32(lbe_handle *h, double *rho_out, double *u_out, double *f_out);
// poisson.cu
cudaError_t poisson_alloc(lbe_handle *h);
void poisson_free(lbe_handle *h);
// enqueue one Poisson solve on the handle's stream (no host synchronisation
// on the graph path)
// extrapolated: the warm start was already applied this step (by the
// advection kernel); only the history count advances
int poisson_enqueue(lbe_handle *h, bool extrapolate, bool extrapolated = false);
// synchronise and read the solves' status/statistics since the last reset;
// *kernels (optional) receives the kernels the graph path launched
int poisson_status(lbe_handle *h, lbe_stats *st, long long *kernels);
// enqueue a solve of A x = rhs on fluid nodes (A = -lap_mod with zero
// Dirichlet values on solid nodes; FP32 form): iterative refinement with an
// FP64 residual from x, stopping when max |res|/diag <= max(tol_abs,
// tol_rel * max |rhs|/diag).  x (FP64, N) is the warm start on entry and
// must hold 0 on solid nodes; rhs (FP64, N) is read on fluid nodes.
// A x = rhs to max(tol_abs, tol_rel max|rhs|/diag) from the given x; with
// x_hi/x_lo (scratch, N floats each) the residual is evaluated in
// float-float arithmetic, which needs every rhs value to be a float
int poisson_solve_linear(lbe_handle *h, const double *rhs, double *x, double tol_abs, double tol_rel,
                         float *x_hi = nullptr, float *x_lo = nullptr);
cudaError_t poisson_reset_stats(lbe_handle *h);
void poisson_drop_graphs(lbe_handle *h);
// lbe_api.cu: message returned by lbe_last_error(NULL) (thread-local)
void set_static_error(const char *msg);
// lbe_api.cu: derived constants (Phys, P32) of h->prm
void fill_constants(lbe_handle *h);
// adjoint.cu
void adjoint_free(lbe_handle *h);
// mg.cu
cudaError_t mg_setup(lbe_handle *h);
void mg_free(lbe_handle *h);
cudaError_t mg_vcycle(lbe_handle *h, const float *r0, float *u0, const PoissonCtl *c, cudaGraph_t gr,
                      cudaGraphNode_t *last, cudaStream_t st);
int mg_kernels_per_cycle(const lbe_handle *h);
// FP32 form: the FP64 potential (set by the API) -> the fixed-point master
// and its float copy, every node (a potential beyond kPhiMax or non-finite
// raises the range flag)
cudaError_t launch_phi_from64(lbe_handle *h);
// FP32 form: the FP64 copy refreshed from the fixed-point master when stale
cudaError_t sync_phi64(lbe_handle *h);
// FP32 form: the float copy from the fixed-point master, every node
cudaError_t launch_phi32_from_fx(lbe_handle *h);
}  // namespace lbe
