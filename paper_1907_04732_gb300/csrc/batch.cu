// Batched FP32 LBE: many independent lattices (instances) of uneven sizes
// advanced together (declarations and contracts in include/lbe.h).
//
// The instances' arrays are concatenated (component stride = total node
// count).  Work is cut into tiles of kTile consecutive nodes of one instance;
// every kernel is a persistent launch whose blocks stride over a tile list,
// so one launch covers all instances whatever their sizes, and a whole step
// is one CUDA graph launch.  The per-node physics is the single-lattice FP32
// code (fp32_device.cuh).
//
// The Poisson solve is the single-lattice iterative refinement with a
// Chronopoulos-Gear CG preconditioned by a multigrid V-cycle (mg_device.cuh),
// batched: every instance has its own scalars, hierarchy and convergence
// test, and the nested device-side while loops run while any instance is
// still working.  Instances converge after different iteration counts, so
// the CG and V-cycle kernels walk only the tiles of instances still
// iterating: after every convergence test the test kernel's last block
// rebuilds, per tile list, the prefix sums of the active instances' tile
// counts, and a block finds the instance of its k-th active tile by binary
// search.  Reductions are per instance and in a fixed order, so results do
// not depend on the launch shape.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <thread>
#include <vector>

#include "fp32_device.cuh"
#include "mg_device.cuh"

constexpr int kBE = LBE_BATCH_MAX_ELECTRODES;  // electrodes per instance

namespace lbe {

// Division of unsigned 32-bit integers by a run-time invariant divisor d >= 1
// by a multiplication and shifts (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, Sec. 4): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// q = (t + ((n - t) >> min(l,1))) >> max(l-1,0), t = high word of m n.
struct FastDiv {
  uint32_t d, m;
  int sh1, sh2;
};

inline FastDiv make_fastdiv(uint32_t d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.d = d;
  f.m = (uint32_t)(((((uint64_t)1 << l) - d) << 32) / d + 1);
  f.sh1 = l < 1 ? l : 1;
  f.sh2 = l > 1 ? l - 1 : 0;
  return f;
}

__host__ __device__ __forceinline__ uint32_t fdiv(const FastDiv &f, uint32_t n) {
#ifdef __CUDA_ARCH__
  const uint32_t t = __umulhi(f.m, n);
#else
  const uint32_t t = (uint32_t)(((uint64_t)f.m * n) >> 32);
#endif
  return (t + ((n - t) >> f.sh1)) >> f.sh2;
}

// host check of a divisor on the values around every multiple boundary that
// matters for indices below nmax, and a spread of others
inline bool fastdiv_ok(const FastDiv &f, uint32_t nmax) {
  const uint32_t d = f.d;
  for (uint64_t k = 0; k * d <= (uint64_t)nmax + d && k < 70000; ++k)
    for (int64_t o = -1; o <= 1; ++o) {
      const int64_t n = (int64_t)(k * d) + o;
      if (n < 0 || n > (int64_t)nmax) continue;
      if (fdiv(f, (uint32_t)n) != (uint32_t)n / d) return false;
    }
  for (uint64_t n = 0; n <= nmax; n += 1 + nmax / 4096)
    if (fdiv(f, (uint32_t)n) != (uint32_t)n / d) return false;
  return true;
}

constexpr int kTile = 1024;           // nodes per tile
constexpr int kSub = kTile / kBlock;  // nodes per thread per tile

struct InstDev {
  Geo g;              // this instance's lattice
  int off;            // first node in the batch arrays
  int tile0, ntiles;  // its tiles in the level-0 tile list
  int n_elec;
  uint32_t selfmask;
  int mg_levels;      // multigrid levels incl. the lattice (0: Jacobi)
  FastDiv fx, fxy;    // division by nx and by nx*ny
  float c6_hi, c6_lo;  // 6 * 4 pi l_B * s (fixed-point unit), as two floats
  double four_pi_lb, eps;
  P32 P;
};

// one multigrid level of one instance: its shape (component stride = the
// level's total node count), first node in the level arrays, first tile in
// the level's tile list, tile count
struct LvSeg {
  mgd::MgLevel L;
  int off, tile0, ntiles;
  FastDiv fx, fxy;  // division by nx and by nx*ny of the level
};

// device arrays of the coarse levels (index = level; 0 unused)
struct LvPtrs {
  float *A[kMaxLevels], *r[kMaxLevels], *e[kMaxLevels];
  float *z[kMaxLevels];  // pre-smoothed iterate omega r/diag
};

struct InstCtl {
  int outer_done, inner_done, solving, rounds, status, pad;
  long long iters;
  double res, res0, alpha, beta, gamma;
};

struct BatchCtl {
  int arrive;
  int sticky_status;
  long long total_iters, solves, max_iters;
  int any_outer, any_inner;  // loop conditions, for the host-polled solve
};

// CG vectors (each Ntot floats)
struct CgVec {
  float *r, *u, *w, *x, *p, *s;
};

}  // namespace lbe

struct lbe_batch {
  int n = 0;
  std::vector<lbe_params> prm;
  std::vector<lbe::InstDev> inst;
  std::vector<std::vector<uint8_t>> ids;
  std::vector<double> psi;  // [n][kBE + 1]
  std::vector<int> have_geometry;
  bool initialised = false;
  bool flow = true;
  long long Ntot = 0;
  int T = 0;  // level-0 tiles
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  std::string err;
  lbe_stats stats{};
  int grid = 0;  // persistent grid (blocks), picked by the autotuner
  double tuned_ms[LBE_BATCH_TUNE_CANDIDATES] = {};
  // device
  lbe::InstDev *inst_d = nullptr;
  int *tile_inst = nullptr;
  uint8_t *id = nullptr;
  uint32_t *mask = nullptr;
  float *f[2] = {nullptr, nullptr};  // populations: f[0], updated in place
  bool aa_odd = false;                // the next step is an odd one of the AA pattern
  int64_t *q = nullptr, *qstar = nullptr;
  double *phi = nullptr;          // FP64 copy of the potential (charges, fields), refreshed when read
  int64_t *phifx = nullptr;       // the potential in fixed point (unit 2^-kPhiFixBits), the master copy
  int64_t *phi_prev = nullptr;    // [kHist][Ntot]: the previous solutions, fixed point
  bool phi64_stale = false;       // phi lags phifx
  float *phi32 = nullptr;         // nearest float of phifx
  float4 *u = nullptr;            // velocity records (fp32::octant_code)
  float4 *lf = nullptr;     // link records, one per node (fp32::link_record)
  float *vec = nullptr;     // CG vectors [6][Ntot]
  double *part = nullptr;   // per-tile partials [3][T]
  double *psi_d = nullptr;  // [n][kBE + 1]
  lbe::InstCtl *ictl = nullptr;
  lbe::BatchCtl *bctl = nullptr, *bctl_h = nullptr;
  double *qpart = nullptr, *qout = nullptr, *qhost = nullptr;
  int *flag = nullptr;
  int *hist = nullptr;  // device: how many solutions phi_prev holds (0..kHist)
  // tile lists of active instances: family f counts, prefix sums
  int nfam = 0;
  int *fam_cnt = nullptr;   // [nfam][n]
  int *fam_pref = nullptr;  // [nfam][n + 1]
  // batched multigrid preconditioner
  int mg_nlev = 0;                       // most levels of any instance
  long long mg_M[lbe::kMaxLevels] = {};  // nodes per coarse level (all instances)
  int mg_T[lbe::kMaxLevels] = {};        // tiles per level
  int mg_tbase[lbe::kMaxLevels] = {};    // level's first entry in mg_tiles
  int *mg_tiles = nullptr;               // tile -> instance, levels 1.. concatenated
  lbe::LvSeg *mg_seg = nullptr;          // [kMaxLevels][n]
  lbe::LvPtrs mg_p{};
  float *mg_t0 = nullptr;
  float *mg_cinv = nullptr;          // inverses of the coarsest operators, concatenated
  long long *mg_cinv_off = nullptr;  // device [n]: an instance's inverse (-1: Jacobi sweeps)
  // step graphs keyed by (in-place step kind, solute read); [4] = solve
  // only; [5..8] step graphs with profiling events
  cudaGraphExec_t exec[9] = {};
  int key_odd[9] = {};
  const void *key_q[9] = {};
  bool polled = false;  // LBE_POISSON_GRAPH=0: solve loops driven by the host
  // profiling (lbe_batch_profile_begin/end): events around the phases
  bool profiling = false;
  cudaEvent_t ev[4] = {};
  double prof_ms[3] = {};
  long long prof_steps = 0, prof_iters = 0, prof_solves = 0, prof_launches = 0;

  lbe::CgVec cg() const {
    const long long N = Ntot;
    return lbe::CgVec{vec, vec + N, vec + 2 * N, vec + 3 * N, vec + 4 * N, vec + 5 * N};
  }
};

namespace lbe {
namespace {

using namespace fp32;
constexpr int kMaxOuterB = 24;

// Families of active-tile lists (index f):
//   f = l           level-l tiles of instances that have level l (l = 0: all)
//   f = nlev + l    level-l tiles of instances that have level l+1
__host__ __device__ constexpr int famA(int l) { return l; }
__host__ __device__ constexpr int famB(int nlev, int l) { return nlev + l; }

// instance-local coordinates of node lo (false past the instance's end)
__device__ __forceinline__ bool node_xyz(const InstDev &I, int lo, int &x, int &y, int &z) {
  if (lo >= I.g.N) return false;
  z = (int)fdiv(I.fxy, (uint32_t)lo);
  const int rem = lo - z * (int)I.fxy.d;
  y = (int)fdiv(I.fx, (uint32_t)rem);
  x = rem - y * I.g.nx;
  return true;
}

// coordinates of node I of a coarse level
__device__ __forceinline__ void lv_xyz(const LvSeg &S, int I, int &X, int &Y, int &Z) {
  Z = (int)fdiv(S.fxy, (uint32_t)I);
  const int rem = I - Z * (int)S.fxy.d;
  Y = (int)fdiv(S.fx, (uint32_t)rem);
  X = rem - Y * S.L.nx;
}

// instance of the tp-th active tile: pref[i] <= tp < pref[i+1]
__device__ __forceinline__ int find_inst(const int *__restrict__ pref, int n, int tp) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pref[mid] <= tp) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, int use, unsigned v) {
  if (use) cudaGraphSetConditional(h, v);
}

template <bool MAX>
__device__ __forceinline__ double breduce(double v) {
  __shared__ double sh[kBlock / 32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_down_sync(0xffffffffu, v, o);
    v = MAX ? fmax(v, u) : v + u;
  }
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double out = 0.0;
  if (t == 0) {
    out = sh[0];
    for (int w = 1; w < kBlock / 32; ++w) out = MAX ? fmax(out, sh[w]) : out + sh[w];
  }
  return out;
}

template <bool MAX>
__device__ __forceinline__ float breducef(float v) {
  __shared__ float sh[kBlock / 32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const float u = __shfl_down_sync(0xffffffffu, v, o);
    v = MAX ? fmaxf(v, u) : v + u;
  }
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  float out = 0.f;
  if (t == 0) {
    out = sh[0];
    for (int w = 1; w < kBlock / 32; ++w) out = MAX ? fmaxf(out, sh[w]) : out + sh[w];
  }
  return out;
}

__device__ __forceinline__ bool last_block(int *arrive, int nblk) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(arrive, 1) == nblk - 1;
  }
  __syncthreads();
  return last;
}

// Prefix sums of the active instances' tile counts for every family; all
// threads of one block (the last block of a convergence-test kernel, after
// every instance's inner_done is final)
__device__ void build_active(const InstCtl *__restrict__ c, int n, int nfam, const int *__restrict__ cnt,
                             int *__restrict__ pref) {
  __shared__ int sc[kBlock];
  const int t = threadIdx.x;
  const int per = (n + kBlock - 1) / kBlock;
  const int i0 = t * per, i1 = min(i0 + per, n);
  for (int f = 0; f < nfam; ++f) {
    const int *cf = cnt + (long long)f * n;
    int *pf = pref + (long long)f * (n + 1);
    int s = 0;
    for (int i = i0; i < i1; ++i) s += __ldcg(&c[i].inner_done) ? 0 : cf[i];
    sc[t] = s;
    __syncthreads();
    for (int o = 1; o < kBlock; o <<= 1) {  // inclusive scan
      const int v = t >= o ? sc[t - o] : 0;
      __syncthreads();
      sc[t] += v;
      __syncthreads();
    }
    int run = t ? sc[t - 1] : 0;
    for (int i = i0; i < i1; ++i) {
      pf[i] = run;
      run += __ldcg(&c[i].inner_done) ? 0 : cf[i];
    }
    if (t == kBlock - 1) pf[n] = sc[t];
    __syncthreads();
  }
}

// --- set-up and step kernels (all level-0 tiles) ------------------------------
__global__ void __launch_bounds__(kBlock) kb_init(const InstDev *__restrict__ inst, const int *__restrict__ tile_inst,
                                                  int T, long long Ntot, const uint8_t *__restrict__ id,
                                                  const double *__restrict__ psi, float *__restrict__ f,
                                                  int64_t *__restrict__ q, double *__restrict__ phi,
                                                  float *__restrict__ phi32, int64_t *__restrict__ phifx,
                                                  int64_t *__restrict__ phi_prev,
                                                  float4 *__restrict__ u) {
  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    const int ii = tile_inst[t];
    const InstDev &I = inst[ii];
    for (int k = 0; k < kSub; ++k) {
      const int lo = (t - I.tile0) * kTile + k * kBlock + threadIdx.x;
      if (lo >= I.g.N) break;
      const long long r = I.off + lo;
      const int e = id[r];
      for (int i = 0; i < kQ; ++i) f[i * Ntot + r] = 0.f;
      for (int s = 0; s < 2; ++s) q[s * Ntot + r] = e ? -(1LL << kFixBits) : 0;
      const double p = e ? psi[ii * (kBE + 1) + e] : 0.0;
      const long long pf = __double2ll_rn(p * 281474976710656.0);  // 2^kPhiFixBits
      phi[r] = p;
      phifx[r] = pf;
      phi32[r] = fx_to_f(pf);
      for (int k = 0; k < kHist; ++k) phi_prev[k * Ntot + r] = pf;
      u[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// link records of every fluid node (fp32::link_record) from the potential
// and solute of the step about to run
__global__ void __launch_bounds__(kBlock) kb_prep(const InstDev *__restrict__ inst, const int *__restrict__ tile_inst,
                                                  int T, int Ntot, const float *__restrict__ phi,
                                                  const int64_t *__restrict__ q, float4 *__restrict__ lf) {
  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    const InstDev &I = inst[tile_inst[t]];
    for (int k = 0; k < kSub; ++k) {
      const int lo = (t - I.tile0) * kTile + k * kBlock + threadIdx.x;
      if (lo >= I.g.N) break;
      const int r = I.off + lo;
      lf[r] = link_record(I.P, phi[r], q[r], q[Ntot + r]);  // solid records are never read
    }
  }
}

// the populations are updated in place (fin == fout; LAYOUT POP_AA_EVEN or
// POP_AA_ODD, the AA pattern of fp32_device.cuh)
template <bool FLOW, int WIDE, int LAYOUT>
__global__ void __launch_bounds__(kBlock, 4) kb_sweep(const InstDev *__restrict__ inst, const int *__restrict__ tile_inst,
                                                   int T, int Ntot, const uint32_t *__restrict__ mask,
                                                   const float *__restrict__ fin, float *__restrict__ fout,
                                                   const int64_t *__restrict__ q, int64_t *__restrict__ qstar,
                                                   const float4 *__restrict__ lf, float4 *__restrict__ u,
                                                   int *__restrict__ flag) {
  // the tile's instance constants are staged in shared memory: the link loop
  // reads them for every link (shared loads instead of global ones)
  __shared__ InstDev sI;
  bool over = false;
  for (int t = blockIdx.x; t < T; t += gridDim.x) {  // the same t for the whole block
    __syncthreads();  // the previous tile's readers are done
    {
      const int *src = reinterpret_cast<const int *>(inst + tile_inst[t]);
      int *dst = reinterpret_cast<int *>(&sI);
      for (int w = threadIdx.x; w < (int)(sizeof(InstDev) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    const InstDev &I = sI;
    for (int k = 0; k < kSub; ++k) {
      int x, y, z;
      const int lo = (t - I.tile0) * kTile + k * kBlock + threadIdx.x;
      if (!node_xyz(I, lo, x, y, z)) break;
      const int r = I.off + lo;
      const uint32_t m = mask[r];
      if (!(m & kFluidBit)) continue;
      sweep_node_lf<FLOW, WIDE, LAYOUT>(I.P, Ntot, r, offsets_of(I.g, x, y, z), m, fin, fout, q, qstar, lf, u,
                                        over);
    }
  }
  if (over) atomicOr(flag, 1);
}

using SweepKern = void (*)(const InstDev *, const int *, int, int, const uint32_t *, const float *, float *,
                          const int64_t *, int64_t *, const float4 *, float4 *, int *);
using PrepKern = void (*)(const InstDev *, const int *, int, int, const float *, const int64_t *, float4 *);
// the sweep for the batch's flow mode, size (the width of the population
// offsets, fp32::pop_idx_kind) and in-place step kind
inline SweepKern sweep_kernel(bool flow, long long Ntot, bool odd) {
  const SweepKern k[3][3] = {
      {kb_sweep<false, 0, POP_AA_EVEN>, kb_sweep<false, 1, POP_AA_EVEN>, kb_sweep<false, 2, POP_AA_EVEN>},
      {kb_sweep<true, 0, POP_AA_EVEN>, kb_sweep<true, 1, POP_AA_EVEN>, kb_sweep<true, 2, POP_AA_EVEN>},
      {kb_sweep<true, 0, POP_AA_ODD>, kb_sweep<true, 1, POP_AA_ODD>, kb_sweep<true, 2, POP_AA_ODD>}};
  return k[flow ? (odd ? 2 : 1) : 0][pop_idx_kind(Ntot)];
}
inline PrepKern prep_kernel(long long) { return kb_prep; }

__global__ void __launch_bounds__(kBlock, 5) kb_advect(const InstDev *__restrict__ inst, const int *__restrict__ tile_inst,
                                                    int T, int Ntot, const uint32_t *__restrict__ mask,
                                                    const int64_t *__restrict__ qin, const float4 *__restrict__ u,
                                                    int64_t *__restrict__ qout, int64_t *__restrict__ phifx,
                                                    int64_t *__restrict__ prev, float *__restrict__ phi32,
                                                    const int *__restrict__ hist) {
  const int have = *hist;  // the next solve's warm start rides along (phi is not read here)
  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    const InstDev &I = inst[tile_inst[t]];
    for (int k = 0; k < kSub; ++k) {
      int x, y, z;
      const int lo = (t - I.tile0) * kTile + k * kBlock + threadIdx.x;
      if (!node_xyz(I, lo, x, y, z)) break;
      const int r = I.off + lo;
      const uint32_t m = mask[r];
      if (!(m & kFluidBit)) {
        qout[r] = qin[r];
        qout[Ntot + r] = qin[Ntot + r];
        continue;
      }
      advect_node2(Ntot, r, offsets_of(I.g, x, y, z), m, qin, u, qout);
      extrapolate_fx(Ntot, r, phifx, prev, phi32, have);
    }
  }
}

// warm start on fluid nodes (all instances) from the *hist previous
// solutions (fp32::extrapolate_fx; with flow, kb_advect does this)
__global__ void kb_extrapolate(const InstDev *__restrict__ inst, const int *__restrict__ tile_inst, int T,
                               int Ntot, const uint32_t *__restrict__ mask, int64_t *__restrict__ phifx,
                               int64_t *__restrict__ prev, float *__restrict__ phi32, const int *__restrict__ hist) {
  const int have = *hist;
  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    const InstDev &I = inst[tile_inst[t]];
    for (int k = 0; k < kSub; ++k) {
      const int lo = (t - I.tile0) * kTile + k * kBlock + threadIdx.x;
      if (lo >= I.g.N) break;
      const int r = I.off + lo;
      if (!(mask[r] & kFluidBit)) continue;
      extrapolate_fx(Ntot, r, phifx, prev, phi32, have);
    }
  }
}

// --- batched Poisson ---------------------------------------------------------
__global__ void kb_solve_reset(int n, InstCtl *c, BatchCtl *b, int *hist, int set_hist) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && set_hist && *hist < kHist) *hist += 1;
  if (i < n) {
    if (c[i].status && !b->sticky_status) b->sticky_status = c[i].status;
    atomicMax((unsigned long long *)&b->max_iters, (unsigned long long)c[i].iters);
    c[i].outer_done = 0;
    c[i].inner_done = 0;
    c[i].solving = 0;
    c[i].rounds = 0;
    c[i].status = 0;
    c[i].iters = 0;
  }
  if (i == 0) b->solves += 1;
}

// Residual (float-float, phi = hi + lo) of the instances still solving;
// seeds their CG (r, u = r/diag, x = p = s = 0); per-tile max |r|/diag
__global__ void __launch_bounds__(kBlock) kb_res(const InstDev *__restrict__ inst, const int *__restrict__ tile_inst,
                                                 int T, int Ntot, const uint32_t *__restrict__ mask,
                                                 const int64_t *__restrict__ qn, const int64_t *__restrict__ phifx,
                                                 const CgVec v,
                                                 double *__restrict__ part, const InstCtl *__restrict__ c) {
  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    const int ii = tile_inst[t];
    if (c[ii].outer_done) continue;  // block-uniform
    const InstDev &I = inst[ii];
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < kSub; ++k) {
      int x, y, z;
      const int lo = (t - I.tile0) * kTile + k * kBlock + threadIdx.x;
      if (!node_xyz(I, lo, x, y, z)) continue;
      const int r = I.off + lo;
      const uint32_t m = mask[r];
      if (!(m & kFluidBit)) {
        v.r[r] = v.u[r] = v.x[r] = v.p[r] = v.s[r] = 0.f;
        continue;
      }
      // 6 res = 6 lap(phi) + 6 (4 pi l_B s)(q+ - q-): 6 lap exact in fixed
      // point, split into float-float and added to the charge term in
      // float-float (as the single lattice's residual)
      const long long L6 = fp32::lap6_fx(I.g, r, x, y, z, m, phifx);
      const float Lh = ll2f(L6);
      const float S = __fmul_rn(Lh, fp32::kPhiUnitF), E = __fmul_rn(ll2f(L6 - f2ll_rn(Lh)), fp32::kPhiUnitF);
      const long long dq = qn[r] - qn[Ntot + r];  // 1:1 salt, one bulk value
      const float dq_hi = ll2f(dq), dq_lo = ll2f(dq - f2ll_rn(dq_hi));
      const float Bv = I.c6_hi * dq_hi;
      const float Be = fmaf(I.c6_hi, dq_hi, -Bv) + (I.c6_hi * dq_lo + I.c6_lo * dq_hi);
      float t6, te6;
      fp32::two_sum(S, Bv, t6, te6);
      const float rf = (t6 + (te6 + (E + Be))) * (1.f / 6.f);
      const float dinv = __fdividef(6.f, (float)mgd::diag6(m, I.selfmask));
      v.r[r] = rf;
      v.u[r] = rf * dinv;
      v.x[r] = v.p[r] = v.s[r] = 0.f;
      mx = fmaxf(mx, finite_or_inf(fabsf(rf) * dinv));
    }
    mx = breducef<true>(mx);
    if (threadIdx.x == 0) part[2LL * T + t] = (double)mx;
  }
}

// per-instance outer test (one block per instance); the last block sets the
// refinement loop's condition (any instance still solving) and rebuilds the
// active-tile lists
__global__ void __launch_bounds__(kBlock) kb_outer(const InstDev *__restrict__ inst, int n, int T,
                                                   const double *__restrict__ part, InstCtl *c, BatchCtl *b,
                                                   double tol, int maxit, int nfam, const int *__restrict__ fam_cnt,
                                                   int *__restrict__ fam_pref, cudaGraphConditionalHandle hout,
                                                   cudaGraphConditionalHandle hin, int use_cond, int set_hin) {
  const int ii = blockIdx.x;
  if (!c[ii].outer_done) {
    const InstDev &I = inst[ii];
    double m = 0.0;
    for (int k = threadIdx.x; k < I.ntiles; k += kBlock) m = fmax(m, __ldcg(part + 2LL * T + I.tile0 + k));
    m = breduce<true>(m);
    if (threadIdx.x == 0) {
      InstCtl &C = c[ii];
      const double prev = C.res;
      C.res = m;
      int done = 0;
      if (m <= tol) done = 1;
      else if (!(m == m) || m > 1e300) { done = 1; C.status = LBE_ERR_NONFINITE; }
      // out of rounds or iterations, or a round that did not halve the
      // residual (the tolerance is below what the arithmetic resolves)
      else if (C.rounds >= kMaxOuterB || C.iters >= maxit || (C.rounds >= 1 && m > 0.5 * prev)) {
        done = 1;
        C.status = LBE_ERR_NOCONVERGE;
      }
      C.outer_done = done;
      C.inner_done = done;
      C.solving = !done;
      C.rounds += 1;
    }
  } else if (threadIdx.x == 0) {
    c[ii].solving = 0;
    c[ii].inner_done = 1;
  }
  if (!last_block(&b->arrive, n)) return;
  if (threadIdx.x == 0) {
    b->arrive = 0;
    int any = 0;
    for (int i = 0; i < n; ++i) any |= !__ldcg(&c[i].outer_done);
    set_cond(hout, use_cond, any ? 1u : 0u);
    if (!any && set_hin) set_cond(hin, use_cond, 0u);
    b->any_outer = any;
    if (!any) b->any_inner = 0;
  }
  build_active(c, n, nfam, fam_cnt, fam_pref);
}

// w = A u (fluid operator) on the active tiles; per-tile partials (r,u), (w,u)
__global__ void __launch_bounds__(kBlock) kb_cg_b(const InstDev *__restrict__ inst, int n, const int *__restrict__ pref,
                                                  int T, const uint32_t *__restrict__ mask,
                                                  const float *__restrict__ r_, const float *__restrict__ u_,
                                                  float *__restrict__ w_, double *__restrict__ part) {
  const int Tact = pref[n];
  for (int tp = blockIdx.x; tp < Tact; tp += gridDim.x) {
    const int ii = find_inst(pref, n, tp);
    const InstDev &I = inst[ii];
    const int j = tp - pref[ii];
    float ru = 0.f, wu = 0.f;
#pragma unroll
    for (int k = 0; k < kSub; ++k) {
      int x, y, z;
      const int lo = j * kTile + k * kBlock + threadIdx.x;
      if (!node_xyz(I, lo, x, y, z)) continue;
      const int r = I.off + lo;
      const uint32_t m = mask[r];
      if (!(m & kFluidBit)) continue;
      const float u0 = u_[r];
      const float s6 = mgd::nbsum6(m, I.selfmask, offsets_of(I.g, x, y, z), r, u_);
      const float wv = ((float)mgd::diag6(m, I.selfmask) * u0 - s6) * (1.f / 6.f);
      w_[r] = wv;
      ru += r_[r] * u0;
      wu += wv * u0;
    }
    ru = breducef<false>(ru);
    wu = breducef<false>(wu);
    if (threadIdx.x == 0) {
      const int t = I.tile0 + j;
      part[t] = (double)ru;
      part[(long long)T + t] = (double)wu;
    }
  }
}

// per-instance scalar recurrence (one block per instance); the last block
// sets the CG loop's condition (any instance still iterating) and rebuilds
// the active-tile lists
__global__ void __launch_bounds__(kBlock) kb_scal(const InstDev *__restrict__ inst, int n, int T,
                                                  const double *__restrict__ part, InstCtl *c, BatchCtl *b,
                                                  double eta, double tol_abs, int maxit, int init, int nfam,
                                                  const int *__restrict__ fam_cnt, int *__restrict__ fam_pref,
                                                  cudaGraphConditionalHandle hin, int use_cond) {
  const int ii = blockIdx.x;
  if (!c[ii].inner_done) {
    const InstDev &I = inst[ii];
    double g = 0.0, d = 0.0, m = 0.0;
    for (int k = threadIdx.x; k < I.ntiles; k += kBlock) {
      g += __ldcg(part + I.tile0 + k);
      d += __ldcg(part + (long long)T + I.tile0 + k);
      if (!init) m = fmax(m, __ldcg(part + 2LL * T + I.tile0 + k));
    }
    g = breduce<false>(g);
    d = breduce<false>(d);
    m = breduce<true>(m);
    if (threadIdx.x == 0) {
      InstCtl &C = c[ii];
      int done = 0;
      if (init) {
        C.res0 = C.res;
        C.beta = 0.0;
        C.alpha = g / d;
        C.gamma = g;
        if (!(d > 0.0) || !(g > 0.0)) done = 1;  // zero residual: nothing to solve
      } else {
        C.iters += 1;
        atomicAdd((unsigned long long *)&b->total_iters, 1ULL);
        if (m <= fmax(eta * C.res0, tol_abs)) done = 1;
        else if (!(m == m) || m > 1e300 || !(d == d)) { done = 1; C.status = LBE_ERR_NONFINITE; C.outer_done = 1; }
        else if (C.iters >= maxit) done = 1;
        else {
          const double beta = g / C.gamma;
          const double den = d - beta * g / C.alpha;
          if (!(den > 0.0) || !(g > 0.0)) done = 1;  // breakdown: converged to rounding
          else { C.beta = beta; C.alpha = g / den; C.gamma = g; }
        }
      }
      C.inner_done = done;
    }
  }
  if (!last_block(&b->arrive, n)) return;
  if (threadIdx.x == 0) {
    b->arrive = 0;
    int any = 0;
    for (int i = 0; i < n; ++i) any |= !__ldcg(&c[i].inner_done);
    set_cond(hin, use_cond, any ? 1u : 0u);
    b->any_inner = any;
  }
  build_active(c, n, nfam, fam_cnt, fam_pref);
}

// p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = r/diag on
// the active tiles; per-tile max |r|/diag
__global__ void __launch_bounds__(kBlock) kb_cg_a(const InstDev *__restrict__ inst, int n, const int *__restrict__ pref,
                                                  int T, const uint32_t *__restrict__ mask, const CgVec v,
                                                  double *__restrict__ part, const InstCtl *__restrict__ c) {
  float *__restrict__ r_ = v.r;
  float *__restrict__ u_ = v.u;
  const float *__restrict__ w_ = v.w;
  float *__restrict__ x_ = v.x;
  float *__restrict__ p_ = v.p;
  float *__restrict__ s_ = v.s;
  const int Tact = pref[n];
  for (int tp = blockIdx.x; tp < Tact; tp += gridDim.x) {
    const int ii = find_inst(pref, n, tp);
    const InstDev &I = inst[ii];
    const int j = tp - pref[ii];
    const float alpha = (float)c[ii].alpha, beta = (float)c[ii].beta;
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < kSub; ++k) {
      const int lo = j * kTile + k * kBlock + threadIdx.x;
      if (lo >= I.g.N) continue;
      const int r = I.off + lo;
      const uint32_t m = mask[r];
      if (!(m & kFluidBit)) continue;
      const float pv = u_[r] + beta * p_[r];
      const float sv = w_[r] + beta * s_[r];
      p_[r] = pv;
      s_[r] = sv;
      x_[r] += alpha * pv;
      const float rv = r_[r] - alpha * sv;
      r_[r] = rv;
      const float dinv = __fdividef(6.f, (float)mgd::diag6(m, I.selfmask));
      u_[r] = rv * dinv;
      mx = fmaxf(mx, finite_or_inf(fabsf(rv) * dinv));
    }
    mx = breducef<true>(mx);
    if (threadIdx.x == 0) part[2LL * T + I.tile0 + j] = (double)mx;
  }
}

// the fixed-point potential += x (rounded to its unit) for instances that
// solved this round, its float copy refreshed; |phi| reaching kPhiMax raises
// range flag 4
__global__ void kb_correct(const InstDev *__restrict__ inst, const int *__restrict__ tile_inst, int T,
                           const uint32_t *__restrict__ mask, const float *__restrict__ x_,
                           int64_t *__restrict__ phifx, float *__restrict__ phi32, int *__restrict__ flag,
                           const InstCtl *__restrict__ c) {
  constexpr float kMaxFx = (float)(kPhiMax * 281474976710656.0);
  bool over = false;
  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    const int ii = tile_inst[t];
    if (!c[ii].solving) continue;
    const InstDev &I = inst[ii];
    for (int k = 0; k < kSub; ++k) {
      const int lo = (t - I.tile0) * kTile + k * kBlock + threadIdx.x;
      if (lo >= I.g.N) break;
      const int r = I.off + lo;
      if (!(mask[r] & kFluidBit)) continue;
      const float d = __fmul_rn(x_[r], 281474976710656.0f);  // x 2^kPhiFixBits, exact
      if (!(fabsf(d) < kMaxFx)) {  // also NaN
        over = true;
        continue;
      }
      const long long v = phifx[r] + f2ll_rn(d);
      over |= !(fabsf(ll2f(v)) < kMaxFx);
      phifx[r] = v;
      phi32[r] = fx_to_f(v);
    }
  }
  if (over) atomicOr(flag, 4);
}

// fixed point -> the FP64 copy, every node of the batch
__global__ void kb_phi_to64(long long Ntot, const int64_t *__restrict__ phifx, double *__restrict__ phi) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < Ntot; r += (long long)gridDim.x * blockDim.x)
    phi[r] = (double)phifx[r] * (1.0 / 281474976710656.0);
}

// induced charge per instance and electrode (Eq. Qelec), FP64, fixed order
__global__ void __launch_bounds__(kBlock) kb_charge(const InstDev *__restrict__ inst, const int *__restrict__ tile_inst,
                                                    int T, const uint8_t *__restrict__ id,
                                                    const uint32_t *__restrict__ mask, const double *__restrict__ phi,
                                                    double *__restrict__ part) {
  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    const InstDev &I = inst[tile_inst[t]];
    double a[kBE];
    for (int e = 0; e < kBE; ++e) a[e] = 0.0;
    for (int k = 0; k < kSub; ++k) {
      int x, y, z;
      const int lo = (t - I.tile0) * kTile + k * kBlock + threadIdx.x;
      if (!node_xyz(I, lo, x, y, z)) break;
      const int r = I.off + lo;
      const int e = id[r];
      const uint32_t m = mask[r];
      if (!e || !(m & ((1u << 18) - 1))) continue;
      const Offs o = offsets_of(I.g, x, y, z);
      double s = 0.0;
      for (int l = 1; l < kQ; ++l)
        if (m & (1u << (l - 1))) s += lapc_of(l) * 2.0 * (phi[r + o.at(cx_of(l), cy_of(l), cz_of(l))] - phi[r]);
      for (int q = 0; q < kBE; ++q)
        if (q == e - 1) a[q] += -I.eps * s;
    }
    for (int q = 0; q < kBE; ++q) {
      const double v = breduce<false>(a[q]);
      if (threadIdx.x == 0) part[(long long)q * T + t] = v;
    }
  }
}

__global__ void kb_charge_final(const InstDev *__restrict__ inst, int T, const double *__restrict__ part,
                                double *__restrict__ q) {
  const int ii = blockIdx.x;
  const InstDev &I = inst[ii];
  for (int k = 0; k < kBE; ++k) {
    double v = 0.0;
    for (int j = threadIdx.x; j < I.ntiles; j += 32) v += part[(long long)k * T + I.tile0 + j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) q[ii * kBE + k] = k < I.n_elec ? v : 0.0;
  }
}

__global__ void kb_n_to_double(const InstDev *__restrict__ inst, int ii, long long Ntot, const int64_t *__restrict__ q,
                               const uint32_t *__restrict__ mask, double *__restrict__ out) {
  const InstDev &I = inst[ii];
  const long long lo = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (lo >= I.g.N) return;
  const long long r = I.off + lo;
  const bool fl = mask[r] & kFluidBit;
  for (int k = 0; k < 2; ++k) out[k * I.g.N + lo] = fl ? I.P.rbd[k] + I.P.sd[k] * (double)q[k * Ntot + r] : 0.0;
}

// --- batched multigrid V-cycle (per-node arithmetic in mg_device.cuh) --------
using mgd::MgLevel;

__global__ void kbm_galerkin0(const InstDev *__restrict__ inst, const int *__restrict__ tiles, int T,
                              const LvSeg *__restrict__ seg1, const uint32_t *__restrict__ mask, float *__restrict__ A1) {
  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    const int ii = tiles[t];
    const LvSeg C = seg1[ii];
    const InstDev &In = inst[ii];
    for (int k = 0; k < kSub; ++k) {
      const int I = (t - C.tile0) * kTile + k * kBlock + threadIdx.x;
      if (I >= C.L.N) break;
      int X, Y, Z;
      lv_xyz(C, I, X, Y, Z);
      float a[27];
      mgd::galerkin0_row(In.g, In.selfmask, mask + In.off, C.L, X, Y, Z, a);
      for (int d = 0; d < 27; ++d) A1[d * C.L.S + C.off + I] = a[d];
    }
  }
}

__global__ void kbm_galerkin(const int *__restrict__ tiles, int T, const LvSeg *__restrict__ segF,
                             const LvSeg *__restrict__ segC, const float *__restrict__ AF, float *__restrict__ AC) {
  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    const int ii = tiles[t];
    const LvSeg C = segC[ii], F = segF[ii];
    for (int k = 0; k < kSub; ++k) {
      const int I = (t - C.tile0) * kTile + k * kBlock + threadIdx.x;
      if (I >= C.L.N) break;
      int X, Y, Z;
      lv_xyz(C, I, X, Y, Z);
      float a[27];
      mgd::galerkin_row(F.L, AF + F.off, C.L, X, Y, Z, a);
      for (int d = 0; d < 27; ++d) AC[d * C.L.S + C.off + I] = a[d];
    }
  }
}

// coarse residual rc and pre-smoothed iterate zc = omega rc/diag of a coarse
// node (lane ch = 0 of its 8)
__device__ __forceinline__ void store_coarse(const LvSeg &C, int I, float v, const float *__restrict__ AC,
                                             float *__restrict__ rc, float *__restrict__ zc) {
  const float d = AC[13 * C.L.S + C.off + I];
  rc[C.off + I] = v;
  zc[C.off + I] = d != 0.f ? mgd::kOmega * v / d : 0.f;
}

// Restriction into level 1 over the active level-1 tiles.  Work item: 32
// coarse nodes, 8 threads each (one per child, fixed-order shuffle sum).  A
// fluid child's pre-smoothed residual is r - omega A u: u = r/diag is the
// Jacobi vector the CG just formed.
__global__ void __launch_bounds__(kBlock) kbm_restrict0(const InstDev *__restrict__ inst, int n,
                                                        const int *__restrict__ pref, const LvSeg *__restrict__ seg1,
                                                        const uint32_t *__restrict__ mask, const float *__restrict__ r,
                                                        const float *__restrict__ u, const float *__restrict__ A1,
                                                        float *__restrict__ rc, float *__restrict__ zc) {
  const int items = pref[n] * (kTile / 32);
  const int ch = threadIdx.x & 7;
  for (int ip = blockIdx.x; ip < items; ip += gridDim.x) {
    const int tp = ip / (kTile / 32);
    const int ii = find_inst(pref, n, tp);
    const LvSeg C = seg1[ii];
    const InstDev &In = inst[ii];
    const int I = (tp - pref[ii]) * kTile + (ip % (kTile / 32)) * 32 + (threadIdx.x >> 3);
    float v = 0.f;
    int X, Y, Z, x, y, z;
    if (I < C.L.N) {
      lv_xyz(C, I, X, Y, Z);
      if (mgd::child_of(C.L, X, Y, Z, ch, In.g.nx, In.g.ny, In.g.nz, x, y, z)) {
        const int i = In.off + x + In.g.nx * (y + In.g.ny * z);
        const uint32_t m = mask[i];
        if (m & kFluidBit) {
          const float s6 = mgd::nbsum6(m, In.selfmask, offsets_of(In.g, x, y, z), i, u);
          v = r[i] - mgd::kOmega * ((float)mgd::diag6(m, In.selfmask) * u[i] - s6) * (1.f / 6.f);
        }
      }
    }
    v = mgd::sum8(v);
    if (ch == 0 && I < C.L.N) store_coarse(C, I, v, A1, rc, zc);
  }
}

// restriction from level l into level l+1 over the active level-(l+1) tiles
__global__ void __launch_bounds__(kBlock) kbm_restrict(int n, const int *__restrict__ pref,
                                                       const LvSeg *__restrict__ segF, const LvSeg *__restrict__ segC,
                                                       const float *__restrict__ AF, const float *__restrict__ rF,
                                                       const float *__restrict__ zF, const float *__restrict__ AC,
                                                       float *__restrict__ rC, float *__restrict__ zC) {
  const int items = pref[n] * (kTile / 32);
  const int ch = threadIdx.x & 7;
  for (int ip = blockIdx.x; ip < items; ip += gridDim.x) {
    const int tp = ip / (kTile / 32);
    const int ii = find_inst(pref, n, tp);
    const LvSeg C = segC[ii], F = segF[ii];
    const int I = (tp - pref[ii]) * kTile + (ip % (kTile / 32)) * 32 + (threadIdx.x >> 3);
    float v = 0.f;
    int X, Y, Z, x, y, z;
    if (I < C.L.N) {
      lv_xyz(C, I, X, Y, Z);
      if (mgd::child_of(C.L, X, Y, Z, ch, F.L.nx, F.L.ny, F.L.nz, x, y, z))
        v = mgd::presmoothed_res_z(F.L, AF + F.off, rF + F.off, zF + F.off, x, y, z);
    }
    v = mgd::sum8(v);
    if (ch == 0 && I < C.L.N) store_coarse(C, I, v, AC, rC, zC);
  }
}

// every instance's coarsest level, one block each: exactly, through the
// inverse formed at set-up (one warp per row, a fixed summation order), or
// by Jacobi sweeps where its operator is not positive definite
__global__ void __launch_bounds__(mgd::kCoarseMax) kbm_coarsest(const InstDev *__restrict__ inst, int n,
                                                                const LvSeg *__restrict__ seg, const LvPtrs P,
                                                                const InstCtl *__restrict__ c,
                                                                const float *__restrict__ cinv,
                                                                const long long *__restrict__ cinv_off) {
  const int ii = blockIdx.x;
  const int nl = inst[ii].mg_levels;
  if (nl < 2 || c[ii].inner_done) return;
  __shared__ float buf[2][mgd::kCoarseMax];
  const LvSeg S = seg[(nl - 1) * n + ii];
  const long long off = cinv_off[ii];
  if (off >= 0) {
    const int N = S.L.N, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const float *r = P.r[nl - 1] + S.off;
    float *e = P.e[nl - 1] + S.off;
    for (int row = threadIdx.x >> 5; row < N; row += nw) {
      const float *a = cinv + off + (long long)row * N;
      float s = 0.f;
      for (int j = lane; j < N; j += 32) s = fmaf(a[j], r[j], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) e[row] = s;
    }
    return;
  }
  mgd::coarsest_solve(S.L, P.A[nl - 1] + S.off, P.r[nl - 1] + S.off, P.e[nl - 1] + S.off, buf);
}

// fused prolongation + post-smoothing on coarse level l over the active
// level-l tiles of instances that have level l+1; work item: 256 nodes
__global__ void __launch_bounds__(kBlock) kbm_post(int n, const int *__restrict__ pref, const LvSeg *__restrict__ segL,
                                                   const LvSeg *__restrict__ segC, const float *__restrict__ A,
                                                   const float *__restrict__ r, const float *__restrict__ z,
                                                   const float *__restrict__ ec, float *__restrict__ e) {
  const int items = pref[n] * kSub;
  for (int ip = blockIdx.x; ip < items; ip += gridDim.x) {
    const int tp = ip / kSub;
    const int ii = find_inst(pref, n, tp);
    const LvSeg L = segL[ii], C = segC[ii];
    const int I = (tp - pref[ii]) * kTile + (ip % kSub) * kBlock + threadIdx.x;
    if (I >= L.L.N) continue;
    int X, Y, Z;
    lv_xyz(L, I, X, Y, Z);
    e[L.off + I] = mgd::post_value_z(L.L, A + L.off, r + L.off, z + L.off, C.L, ec + C.off, X, Y, Z);
  }
}

// level 0 over the active tiles of instances with a hierarchy:
// t = omega u + alpha P e_1 (u = r/diag, the Jacobi vector)
__global__ void __launch_bounds__(kBlock) kbm_prolong0(const InstDev *__restrict__ inst, int n,
                                                       const int *__restrict__ pref, const LvSeg *__restrict__ seg1,
                                                       const uint32_t *__restrict__ mask, const float *__restrict__ u,
                                                       const float *__restrict__ e1, float *__restrict__ t0) {
  const int Tact = pref[n];
  for (int tp = blockIdx.x; tp < Tact; tp += gridDim.x) {
    const int ii = find_inst(pref, n, tp);
    const InstDev &I = inst[ii];
    const LvSeg C = seg1[ii];
    const int j = tp - pref[ii];
#pragma unroll
    for (int k = 0; k < kSub; ++k) {
      int x, y, z;
      const int lo = j * kTile + k * kBlock + threadIdx.x;
      if (!node_xyz(I, lo, x, y, z)) continue;
      const int rr = I.off + lo;
      t0[rr] = (mask[rr] & kFluidBit) ? fmaf(mgd::kAlpha, e1[C.off + mgd::agg_index(C.L, x, y, z)], mgd::kOmega * u[rr])
                                      : 0.f;
    }
  }
}

// then u = t + omega (r - A t)/diag
__global__ void __launch_bounds__(kBlock) kbm_post0(const InstDev *__restrict__ inst, int n,
                                                    const int *__restrict__ pref, const uint32_t *__restrict__ mask,
                                                    const float *__restrict__ r, const float *__restrict__ t0,
                                                    float *__restrict__ u) {
  const int Tact = pref[n];
  for (int tp = blockIdx.x; tp < Tact; tp += gridDim.x) {
    const int ii = find_inst(pref, n, tp);
    const InstDev &I = inst[ii];
    const int j = tp - pref[ii];
#pragma unroll
    for (int k = 0; k < kSub; ++k) {
      int x, y, z;
      const int lo = j * kTile + k * kBlock + threadIdx.x;
      if (!node_xyz(I, lo, x, y, z)) continue;
      const int i = I.off + lo;
      const uint32_t m = mask[i];
      if (!(m & kFluidBit)) {
        u[i] = 0.f;
        continue;
      }
      const float d6 = (float)mgd::diag6(m, I.selfmask);
      const float s6 = mgd::nbsum6(m, I.selfmask, offsets_of(I.g, x, y, z), i, t0);
      const float ti = t0[i];
      u[i] = ti + mgd::kOmega * __fdividef(6.f * r[i] - (d6 * ti - s6), d6);
    }
  }
}

}  // namespace
}  // namespace lbe

// =============================================================================
namespace {

using lbe::kTile;

int bfail(lbe_batch *b, int code, const std::string &m) {
  if (b) b->err = m;
  return code;
}
#define BCK(b, expr)                                                                                  \
  do {                                                                                                \
    cudaError_t e_ = (expr);                                                                          \
    if (e_ != cudaSuccess) return bfail((b), LBE_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void mg_release(lbe_batch *b) {
  cudaFree(b->mg_tiles);
  cudaFree(b->mg_seg);
  cudaFree(b->mg_t0);
  cudaFree(b->mg_cinv);
  cudaFree(b->mg_cinv_off);
  cudaFree(b->fam_cnt);
  cudaFree(b->fam_pref);
  for (int l = 0; l < lbe::kMaxLevels; ++l) {
    cudaFree(b->mg_p.A[l]);
    cudaFree(b->mg_p.r[l]);
    cudaFree(b->mg_p.e[l]);
    cudaFree(b->mg_p.z[l]);
  }
  b->mg_tiles = nullptr;
  b->mg_seg = nullptr;
  b->mg_t0 = nullptr;
  b->mg_cinv = nullptr;
  b->mg_cinv_off = nullptr;
  b->fam_cnt = b->fam_pref = nullptr;
  b->mg_p = lbe::LvPtrs{};
  b->mg_nlev = 0;
  b->nfam = 0;
}

void bfree(lbe_batch *b) {
  void *ptrs[] = {b->inst_d, b->tile_inst, b->id,   b->mask, b->f[0],  b->f[1], b->q,    b->qstar, b->phi,
                  b->phi_prev, b->phi32,  b->phifx, b->u, b->vec, b->part, b->psi_d, b->ictl, b->bctl, b->qpart,
                  b->qout,
                  b->flag,     b->hist,   b->lf};
  for (void *p : ptrs) cudaFree(p);
  mg_release(b);
  if (b->bctl_h) cudaFreeHost(b->bctl_h);
  if (b->qhost) cudaFreeHost(b->qhost);
  for (int k = 0; k < 9; ++k)
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
  for (int k = 0; k < 4; ++k)
    if (b->ev[k]) cudaEventDestroy(b->ev[k]);
}

cudaError_t add_node(cudaGraph_t gr, cudaGraphNode_t *last, void *func, dim3 grid, dim3 block, void **args) {
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof(kp));
  kp.func = func;
  kp.gridDim = grid;
  kp.blockDim = block;
  kp.kernelParams = args;
  cudaGraphNode_t n;
  cudaError_t e = cudaGraphAddKernelNode(&n, gr, *last ? last : nullptr, *last ? 1 : 0, &kp);
  if (e == cudaSuccess) *last = n;
  return e;
}

cudaError_t add_while(cudaGraph_t gr, cudaGraphNode_t *last, cudaGraphConditionalHandle h, cudaGraph_t *body) {
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams *np = reinterpret_cast<cudaGraphNodeParams *>(raw);
  np->type = cudaGraphNodeTypeConditional;
  np->conditional.handle = h;
  np->conditional.type = cudaGraphCondTypeWhile;
  np->conditional.size = 1;
  cudaGraphNode_t n;
  cudaError_t e = cudaGraphAddNode(&n, gr, *last ? last : nullptr, nullptr, *last ? 1 : 0, np);
  if (e == cudaSuccess) {
    *last = n;
    *body = np->conditional.phGraph_out[0];
  }
  return e;
}

cudaError_t add_event(cudaGraph_t gr, cudaGraphNode_t *last, cudaEvent_t ev) {
  cudaGraphNode_t n;
  cudaError_t e = cudaGraphAddEventRecordNode(&n, gr, *last ? last : nullptr, *last ? 1 : 0, ev);
  if (e == cudaSuccess) *last = n;
  return e;
}

// family prefix array f
const int *fam(const lbe_batch *b, int f) { return b->fam_pref + (size_t)f * (b->n + 1); }
int fam_levels(const lbe_batch *b) { return b->mg_nlev >= 2 ? b->mg_nlev : 1; }

// Multigrid hierarchy of every instance (after the link masks): level shapes
// per instance, the levels' concatenated arrays and tile lists, the active-
// Exact coarsest solves: each instance's coarsest operator comes back to the
// host, is inverted there (mgd::coarse_inverse, FP64 Cholesky; instances in
// parallel threads) and the inverses go to the device concatenated.  An
// instance whose operator is not positive definite keeps the Jacobi sweeps
// (offset -1), as does every instance with LBE_MG_DIRECT=0.
int coarse_inverses(lbe_batch *b, const std::vector<lbe::LvSeg> &seg) {
  using namespace lbe;
  const int n = b->n, L = b->mg_nlev;
  std::vector<long long> off(n, -1);
  const char *denv = getenv("LBE_MG_DIRECT");
  const bool direct = !(denv && denv[0] == '0');
  std::vector<std::vector<float>> inv(n);
  if (direct) {
    std::vector<std::vector<float>> Ah(L);
    for (int i = 0; i < n; ++i) {
      const int l = b->inst[i].mg_levels - 1;
      if (l >= 1 && Ah[l].empty()) {
        Ah[l].resize((size_t)27 * b->mg_M[l]);
        BCK(b, cudaMemcpyAsync(Ah[l].data(), b->mg_p.A[l], sizeof(float) * Ah[l].size(), cudaMemcpyDeviceToHost,
                               b->stream));
      }
    }
    BCK(b, cudaStreamSynchronize(b->stream));
    std::vector<char> ok(n, 0);
    auto work = [&](int t, int nt) {
      for (int i = t; i < n; i += nt) {
        const int l = b->inst[i].mg_levels - 1;
        if (l < 1) continue;
        const LvSeg &S = seg[(size_t)l * n + i];
        mgd::MgLevel Lc = S.L;
        Lc.S = Lc.N;
        std::vector<float> a27((size_t)27 * Lc.N);
        for (int q = 0; q < 27; ++q)
          for (int I = 0; I < Lc.N; ++I) a27[(size_t)q * Lc.N + I] = Ah[l][(size_t)q * S.L.S + S.off + I];
        ok[i] = mgd::coarse_inverse(Lc, a27, inv[i]) ? 1 : 0;
      }
    };
    const int nt = std::max(1, std::min<int>(n, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(work, t, nt);
    work(0, nt);
    for (auto &t : th) t.join();
    long long tot = 0;
    for (int i = 0; i < n; ++i)
      if (ok[i]) {
        off[i] = tot;
        tot += (long long)inv[i].size();
      }
    if (tot > 0) {
      BCK(b, cudaMalloc(&b->mg_cinv, sizeof(float) * tot));
      for (int i = 0; i < n; ++i)
        if (ok[i])
          BCK(b, cudaMemcpyAsync(b->mg_cinv + off[i], inv[i].data(), sizeof(float) * inv[i].size(),
                                 cudaMemcpyHostToDevice, b->stream));
    }
  }
  BCK(b, cudaMalloc(&b->mg_cinv_off, sizeof(long long) * n));
  BCK(b, cudaMemcpyAsync(b->mg_cinv_off, off.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));  // the host buffers are released on return
  return LBE_OK;
}

// tile families, then the inverse fine diagonal and the Galerkin operators on
// the GPU.  Uploads the instance table (it carries each instance's level
// count).
int mg_setup(lbe_batch *b) {
  using namespace lbe;
  mg_release(b);
  const int n = b->n;
  std::vector<mgd::MgLevel> shp((size_t)n * kMaxLevels);
  int L = 0;
  for (int i = 0; i < n; ++i) {
    const Geo &g = b->inst[i].g;
    b->inst[i].mg_levels = mgd::level_shapes(g.nx, g.ny, g.nz, &shp[(size_t)i * kMaxLevels]);
    L = std::max(L, b->inst[i].mg_levels);
  }
  b->mg_nlev = L;
  BCK(b, cudaMemcpyAsync(b->inst_d, b->inst.data(), sizeof(InstDev) * n, cudaMemcpyHostToDevice, b->stream));
  std::vector<LvSeg> seg((size_t)kMaxLevels * n);
  memset(seg.data(), 0, sizeof(LvSeg) * seg.size());
  std::vector<int> tiles;
  for (int l = 1; l < L; ++l) {
    b->mg_tbase[l] = (int)tiles.size();
    long long M = 0;
    int T = 0;
    for (int i = 0; i < n; ++i) {
      if (b->inst[i].mg_levels <= l) continue;
      LvSeg &S = seg[(size_t)l * n + i];
      S.L = shp[(size_t)i * kMaxLevels + l];
      S.off = (int)M;
      S.tile0 = T;
      S.ntiles = (S.L.N + kTile - 1) / kTile;
      S.fx = make_fastdiv((uint32_t)S.L.nx);
      S.fxy = make_fastdiv((uint32_t)(S.L.nx * S.L.ny));
      if (!fastdiv_ok(S.fx, (uint32_t)S.L.N) || !fastdiv_ok(S.fxy, (uint32_t)S.L.N))
        return bfail(b, LBE_ERR_STATE, "batch: index division check failed");
      for (int k = 0; k < S.ntiles; ++k) tiles.push_back(i);
      M += S.L.N;
      T += S.ntiles;
    }
    for (int i = 0; i < n; ++i) seg[(size_t)l * n + i].L.S = M;  // component stride
    b->mg_M[l] = M;
    b->mg_T[l] = T;
  }
  // active-tile families
  const int FL = fam_levels(b);
  b->nfam = 2 * FL - 1;
  std::vector<int> cnt((size_t)b->nfam * n, 0);
  for (int i = 0; i < n; ++i) {
    const int ml = b->inst[i].mg_levels;
    auto tiles_at = [&](int l) { return l == 0 ? b->inst[i].ntiles : seg[(size_t)l * n + i].ntiles; };
    for (int l = 0; l < FL; ++l) cnt[(size_t)famA(l) * n + i] = (l == 0 || ml > l) ? tiles_at(l) : 0;
    for (int l = 0; l + 1 < FL; ++l) cnt[(size_t)famB(FL, l) * n + i] = ml > l + 1 ? tiles_at(l) : 0;
  }
  cudaError_t e = cudaMalloc(&b->fam_cnt, sizeof(int) * cnt.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->fam_pref, sizeof(int) * (size_t)b->nfam * (n + 1));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->fam_cnt, cnt.data(), sizeof(int) * cnt.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->fam_pref, 0, sizeof(int) * (size_t)b->nfam * (n + 1), b->stream);
  BCK(b, e);
  if (L < 2) return LBE_OK;
  e = cudaMalloc(&b->mg_tiles, sizeof(int) * std::max<size_t>(tiles.size(), 1));
  if (e == cudaSuccess) e = cudaMalloc(&b->mg_seg, sizeof(LvSeg) * seg.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->mg_t0, sizeof(float) * b->Ntot);
  for (int l = 1; l < L && e == cudaSuccess; ++l) {
    e = cudaMalloc(&b->mg_p.A[l], sizeof(float) * 27 * b->mg_M[l]);
    if (e == cudaSuccess) e = cudaMalloc(&b->mg_p.r[l], sizeof(float) * b->mg_M[l]);
    if (e == cudaSuccess) e = cudaMalloc(&b->mg_p.e[l], sizeof(float) * b->mg_M[l]);
    if (e == cudaSuccess) e = cudaMalloc(&b->mg_p.z[l], sizeof(float) * b->mg_M[l]);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->mg_tiles, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->mg_seg, seg.data(), sizeof(LvSeg) * seg.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->mg_t0, 0, sizeof(float) * b->Ntot, b->stream);
  BCK(b, e);
  const int G = b->grid;
  kbm_galerkin0<<<std::min(G, b->mg_T[1]), kBlock, 0, b->stream>>>(b->inst_d, b->mg_tiles + b->mg_tbase[1],
                                                                   b->mg_T[1], b->mg_seg + n, b->mask,
                                                                   b->mg_p.A[1]);
  for (int l = 1; l + 1 < L; ++l)
    kbm_galerkin<<<std::min(G, b->mg_T[l + 1]), kBlock, 0, b->stream>>>(
        b->mg_tiles + b->mg_tbase[l + 1], b->mg_T[l + 1], b->mg_seg + (size_t)l * n, b->mg_seg + (size_t)(l + 1) * n,
        b->mg_p.A[l], b->mg_p.A[l + 1]);
  BCK(b, cudaGetLastError());
  return coarse_inverses(b, seg);
}

// Blocks of a persistent kernel other than the sweep: the tuned grid, but at
// most as many as the GPU holds at once at the kernel's own occupancy.  A
// block beyond that would start only when a resident one had finished its
// whole share of the tiles, and the kernel would take up to twice as long
// (the coarse levels' post-smoothing, at 64 registers, holds four blocks per
// SM; the tuned grid can have eight).  On the 256-instance sweep: solve 49.7
// -> 47.3 ms per step.  The advection (48 registers) measured no better
// capped (9.29 against 9.14 ms) and keeps the tuned grid, as the sweep.
int resident_grid(const lbe_batch *b, const void *kernel) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0 ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, lbe::kBlock, 0) != cudaSuccess ||
      per_sm <= 0) {
    cudaGetLastError();  // clear; the tuned grid
    return b->grid;
  }
  return std::min(b->grid, per_sm * sms);
}

// u = M r (one V-cycle over every active instance with a hierarchy) as graph
// nodes after *last; r and u are the CG vectors
cudaError_t add_vcycle(lbe_batch *b, cudaGraph_t gr, cudaGraphNode_t *last) {
  using namespace lbe;
  const int L = b->mg_nlev;
  if (L < 2) return cudaSuccess;
  int n = b->n;
  const InstDev *inst = b->inst_d;
  const InstCtl *c = b->ictl;
  const uint32_t *mask = b->mask;
  const CgVec v = b->cg();
  const float *r0 = v.r, *uj = v.u;
  float *u0 = v.u, *t0 = b->mg_t0;
  const LvSeg *seg_all = b->mg_seg;
  LvPtrs P = b->mg_p;
  const dim3 G(b->grid), B(kBlock);
  cudaError_t e;
  {
    const int *pref = fam(b, famA(1));
    const LvSeg *seg1 = seg_all + n;
    const float *A1 = P.A[1];
    float *rc = P.r[1], *zc = P.z[1];
    void *a[] = {&inst, &n, &pref, &seg1, &mask, &r0, &uj, &A1, &rc, &zc};
    e = add_node(gr, last, (void *)kbm_restrict0, dim3(resident_grid(b, (void *)kbm_restrict0)), B, a);
    if (e != cudaSuccess) return e;
  }
  for (int l = 1; l + 1 < L; ++l) {
    const int *pref = fam(b, famA(l + 1));
    const LvSeg *sf = seg_all + (size_t)l * n, *sc = seg_all + (size_t)(l + 1) * n;
    const float *AF = P.A[l], *rF = P.r[l], *zF = P.z[l], *AC = P.A[l + 1];
    float *rC = P.r[l + 1], *zC = P.z[l + 1];
    void *a[] = {&n, &pref, &sf, &sc, &AF, &rF, &zF, &AC, &rC, &zC};
    e = add_node(gr, last, (void *)kbm_restrict, dim3(resident_grid(b, (void *)kbm_restrict)), B, a);
    if (e != cudaSuccess) return e;
  }
  {
    const float *cinv = b->mg_cinv;
    const long long *cinv_off = b->mg_cinv_off;
    void *a[] = {&inst, &n, &seg_all, &P, &c, &cinv, &cinv_off};
    e = add_node(gr, last, (void *)kbm_coarsest, dim3(n), dim3(mgd::kCoarseMax), a);
    if (e != cudaSuccess) return e;
  }
  for (int l = L - 2; l >= 1; --l) {
    const int *pref = fam(b, famB(L, l));
    const LvSeg *sl = seg_all + (size_t)l * n, *sc = seg_all + (size_t)(l + 1) * n;
    const float *A = P.A[l], *r = P.r[l], *z = P.z[l], *ec = P.e[l + 1];
    float *el = P.e[l];
    void *a[] = {&n, &pref, &sl, &sc, &A, &r, &z, &ec, &el};
    e = add_node(gr, last, (void *)kbm_post, dim3(resident_grid(b, (void *)kbm_post)), B, a);
    if (e != cudaSuccess) return e;
  }
  const int *prefB0 = fam(b, famB(L, 0));
  {
    const LvSeg *seg1 = seg_all + n;
    const float *e1 = P.e[1];
    void *a[] = {&inst, &n, &prefB0, &seg1, &mask, &uj, &e1, &t0};
    e = add_node(gr, last, (void *)kbm_prolong0, dim3(resident_grid(b, (void *)kbm_prolong0)), B, a);
    if (e != cudaSuccess) return e;
  }
  {
    const float *tc = t0;
    void *a[] = {&inst, &n, &prefB0, &mask, &r0, &tc, &u0};
    e = add_node(gr, last, (void *)kbm_post0, dim3(resident_grid(b, (void *)kbm_post0)), B, a);
  }
  return e;
}

// kernels of one V-cycle
int vcycle_kernels(const lbe_batch *b) { return b->mg_nlev >= 2 ? 2 * (b->mg_nlev - 1) + 2 : 0; }

// Arguments of the solve kernels (kept alive while nodes are created or
// kernels launched)
struct SolveArgs {
  const lbe::InstDev *inst;
  const int *tile_inst, *pref0, *fam_cnt;
  int T, Ntot, n, maxit, nfam, use = 1, init1 = 1, init0 = 0, set_hist, hin_no = 0, hin_yes = 1;
  const uint32_t *mask;
  const float *fin;
  float *fout;
  int64_t *qin, *qmid, *qsolve;
  int64_t *phifx, *phi_prev;
  float *phi32;
  float4 *u, *lf;
  lbe::CgVec v;
  const float *vr, *vu, *vx;
  float *vw;
  double *part;
  lbe::InstCtl *c;
  lbe::BatchCtl *bc;
  int *flag, *hist, *fam_pref;
  double tol, eta, tol_abs;
  cudaGraphConditionalHandle hout = 0, hin = 0;
};

void solve_args(lbe_batch *b, bool step, const float *fin, float *fout, int64_t *qin, int64_t *qmid, SolveArgs &A) {
  A.inst = b->inst_d;
  A.tile_inst = b->tile_inst;
  A.pref0 = fam(b, lbe::famA(0));
  A.fam_cnt = b->fam_cnt;
  A.fam_pref = b->fam_pref;
  A.T = b->T;
  A.Ntot = (int)b->Ntot;
  A.n = b->n;
  A.nfam = b->nfam;
  A.maxit = b->prm[0].poisson_max_iter;
  A.set_hist = step ? 1 : 0;
  A.mask = b->mask;
  A.fin = fin;
  A.fout = fout;
  A.qin = qin;
  A.qmid = qmid;
  // the solve reads the solute after the step: advected back into qin with
  // flow, the flux-updated copy without
  A.qsolve = !step ? qin : (b->flow ? qin : qmid);
  A.phifx = b->phifx;
  A.phi_prev = b->phi_prev;
  A.phi32 = b->phi32;
  A.u = b->u;
  A.lf = b->lf;
  A.v = b->cg();
  A.vr = A.v.r;
  A.vu = A.v.u;
  A.vx = A.v.x;
  A.vw = A.v.w;
  A.part = b->part;
  A.c = b->ictl;
  A.bc = b->bctl;
  A.flag = b->flag;
  A.hist = b->hist;
  A.tol = b->prm[0].poisson_tol;
  A.eta = 1e-4;
  A.tol_abs = 0.8 * A.tol;  // as the single-lattice solve (fewer CG iterations, same outer test)
}

// One graph per step: [sweep -> advect ->] extrapolate -> Poisson solve
// (nested while loops: refinement rounds around the CG iterations).  With
// step = false only the solve (set-up).
cudaError_t build_graph(lbe_batch *b, bool step, const float *fin, float *fout, int64_t *qin, int64_t *qmid,
                        cudaGraphExec_t *exec, bool prof = false) {
  using namespace lbe;
  SolveArgs A;
  solve_args(b, step, fin, fout, qin, qmid, A);
  const dim3 G(b->grid), B(kBlock), NB(b->n), rb((b->n + 255) / 256);
  // the sweep and the advection take the tuned grid, the other persistent
  // kernels at most one resident wave each (resident_grid)
  const dim3 Gprep(resident_grid(b, (void *)prep_kernel(b->Ntot))), Gadv(b->grid),
      Gext(resident_grid(b, (void *)kb_extrapolate)), Gres(resident_grid(b, (void *)kb_res)),
      Gb(resident_grid(b, (void *)kb_cg_b)), Ga(resident_grid(b, (void *)kb_cg_a)),
      Gcor(resident_grid(b, (void *)kb_correct));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  cudaGraphNode_t last = nullptr, lo = nullptr, li = nullptr;
  cudaGraph_t bo = nullptr, bi = nullptr;
  void *a_prep[] = {&A.inst, &A.tile_inst, &A.T, &A.Ntot, &A.phi32, &A.qin, &A.lf};
  void *a_sw[] = {&A.inst, &A.tile_inst, &A.T, &A.Ntot, &A.mask, &A.fin, &A.fout, &A.qin, &A.qmid, &A.lf, &A.u,
                  &A.flag};
  void *a_adv[] = {&A.inst, &A.tile_inst, &A.T,     &A.Ntot,     &A.mask,  &A.qmid,
                   &A.u,    &A.qin,       &A.phifx, &A.phi_prev, &A.phi32, &A.hist};
  void *a_ext[] = {&A.inst, &A.tile_inst, &A.T, &A.Ntot, &A.mask, &A.phifx, &A.phi_prev, &A.phi32, &A.hist};
  void *a_reset[] = {&A.n, &A.c, &A.bc, &A.hist, &A.set_hist};
  void *a_res[] = {&A.inst, &A.tile_inst, &A.T, &A.Ntot, &A.mask, &A.qsolve, &A.phifx, &A.v, &A.part, &A.c};
  // the test before the round loop must not touch the inner loop's
  // condition (it belongs to the loop body); the one closing a round does
  void *a_out0[] = {&A.inst, &A.n,    &A.T,       &A.part,     &A.c,    &A.bc,  &A.tol,
                    &A.maxit, &A.nfam, &A.fam_cnt, &A.fam_pref, &A.hout, &A.hin, &A.use, &A.hin_no};
  void *a_out[] = {&A.inst, &A.n,    &A.T,       &A.part,     &A.c,    &A.bc,  &A.tol,
                   &A.maxit, &A.nfam, &A.fam_cnt, &A.fam_pref, &A.hout, &A.hin, &A.use, &A.hin_yes};
  void *a_b[] = {&A.inst, &A.n, &A.pref0, &A.T, &A.mask, &A.vr, &A.vu, &A.vw, &A.part};
  void *a_si[] = {&A.inst, &A.n,     &A.T,    &A.part,    &A.c,        &A.bc,  &A.eta, &A.tol_abs,
                  &A.maxit, &A.init1, &A.nfam, &A.fam_cnt, &A.fam_pref, &A.hin, &A.use};
  void *a_st[] = {&A.inst, &A.n,     &A.T,    &A.part,    &A.c,        &A.bc,  &A.eta, &A.tol_abs,
                  &A.maxit, &A.init0, &A.nfam, &A.fam_cnt, &A.fam_pref, &A.hin, &A.use};
  void *a_a[] = {&A.inst, &A.n, &A.pref0, &A.T, &A.mask, &A.v, &A.part, &A.c};
  void *a_cor[] = {&A.inst, &A.tile_inst, &A.T, &A.mask, &A.vx, &A.phifx, &A.phi32, &A.flag, &A.c};
  if (step) {
    void *sweep = (void *)sweep_kernel(b->flow, b->Ntot, b->aa_odd);
    if (prof) e = add_event(g, &last, b->ev[0]);
    if (e == cudaSuccess) e = add_node(g, &last, (void *)prep_kernel(b->Ntot), Gprep, B, a_prep);
    if (e == cudaSuccess) e = add_node(g, &last, sweep, G, B, a_sw);
    if (e == cudaSuccess && prof) e = add_event(g, &last, b->ev[1]);
    if (e == cudaSuccess && b->flow) e = add_node(g, &last, (void *)kb_advect, Gadv, B, a_adv);
    if (e == cudaSuccess && prof) e = add_event(g, &last, b->ev[2]);
    // with flow the advection applies the warm start (kb_advect)
    if (e == cudaSuccess && !b->flow) e = add_node(g, &last, (void *)kb_extrapolate, Gext, B, a_ext);
  }
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&A.hout, g, 1, cudaGraphCondAssignDefault);
  // reset -> residual test -> while (any instance unconverged) { V-cycle ->
  // CG -> correct -> residual test }
  if (e == cudaSuccess) e = add_node(g, &last, (void *)kb_solve_reset, rb, dim3(256), a_reset);
  if (e == cudaSuccess) e = add_node(g, &last, (void *)kb_res, Gres, B, a_res);
  if (e == cudaSuccess) e = add_node(g, &last, (void *)kb_outer, NB, B, a_out0);
  if (e == cudaSuccess) e = add_while(g, &last, A.hout, &bo);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&A.hin, bo, 0, 0);
  if (e == cudaSuccess) e = add_vcycle(b, bo, &lo);
  if (e == cudaSuccess) e = add_node(bo, &lo, (void *)kb_cg_b, Gb, B, a_b);
  if (e == cudaSuccess) e = add_node(bo, &lo, (void *)kb_scal, NB, B, a_si);
  if (e == cudaSuccess) e = add_while(bo, &lo, A.hin, &bi);
  if (e == cudaSuccess) e = add_node(bi, &li, (void *)kb_cg_a, Ga, B, a_a);
  if (e == cudaSuccess) e = add_vcycle(b, bi, &li);
  if (e == cudaSuccess) e = add_node(bi, &li, (void *)kb_cg_b, Gb, B, a_b);
  if (e == cudaSuccess) e = add_node(bi, &li, (void *)kb_scal, NB, B, a_st);
  if (e == cudaSuccess) e = add_node(bo, &lo, (void *)kb_correct, Gcor, B, a_cor);
  if (e == cudaSuccess) e = add_node(bo, &lo, (void *)kb_res, Gres, B, a_res);
  if (e == cudaSuccess) e = add_node(bo, &lo, (void *)kb_outer, NB, B, a_out);
  if (e == cudaSuccess && prof) e = add_event(g, &last, b->ev[3]);
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  return e;
}

void drop_graphs(lbe_batch *b) {
  for (int k = 0; k < 9; ++k) {
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]), b->exec[k] = nullptr;
    b->key_odd[k] = 0;
    b->key_q[k] = nullptr;
  }
}

// The same step with every kernel launched from the host and the solve's
// loop conditions read back after each test (LBE_POISSON_GRAPH=0: lets a
// kernel profiler see the individual launches).
int run_polled(lbe_batch *b, bool step, const float *fin, float *fout, int64_t *qin, int64_t *qmid) {
  using namespace lbe;
  SolveArgs A;
  solve_args(b, step, fin, fout, qin, qmid, A);
  cudaStream_t st = b->stream;
  const int G = b->grid, n = b->n;
  const int Gprep = resident_grid(b, (void *)prep_kernel(b->Ntot)), Gadv = G,
            Gext = resident_grid(b, (void *)kb_extrapolate), Gres = resident_grid(b, (void *)kb_res),
            Gb = resident_grid(b, (void *)kb_cg_b), Ga = resident_grid(b, (void *)kb_cg_a),
            Gcor = resident_grid(b, (void *)kb_correct);
  auto rec = [&](int k) { return b->profiling && step ? cudaEventRecord(b->ev[k], st) : cudaSuccess; };
  long long &nl = b->prof_launches;
  if (step) {
    BCK(b, rec(0));
    prep_kernel(b->Ntot)<<<Gprep, kBlock, 0, st>>>(A.inst, A.tile_inst, A.T, A.Ntot, A.phi32, qin, A.lf);
    sweep_kernel(b->flow, b->Ntot, b->aa_odd)<<<G, kBlock, 0, st>>>(A.inst, A.tile_inst, A.T, A.Ntot, A.mask, fin,
                                                                    fout, qin, qmid, A.lf, A.u, A.flag);
    BCK(b, rec(1));
    if (b->flow)  // the advection applies the warm start as well
      kb_advect<<<Gadv, kBlock, 0, st>>>(A.inst, A.tile_inst, A.T, A.Ntot, A.mask, qmid, A.u, qin, A.phifx, A.phi_prev,
                                      A.phi32, A.hist);
    BCK(b, rec(2));
    if (!b->flow)
      kb_extrapolate<<<Gext, kBlock, 0, st>>>(A.inst, A.tile_inst, A.T, A.Ntot, A.mask, A.phifx, A.phi_prev, A.phi32,
                                           A.hist);
    nl += 3;
  }
  kb_solve_reset<<<(n + 255) / 256, 256, 0, st>>>(n, A.c, A.bc, A.hist, A.set_hist);
  nl += 1;
  // the V-cycle through a small graph keeps it identical to the graph path
  cudaGraphExec_t vc = nullptr;
  if (b->mg_nlev >= 2) {
    cudaGraph_t g;
    BCK(b, cudaGraphCreate(&g, 0));
    cudaGraphNode_t last = nullptr;
    cudaError_t e = add_vcycle(b, g, &last);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&vc, g, 0);
    cudaGraphDestroy(g);
    BCK(b, e);
  }
  const int vck = vcycle_kernels(b);
  cudaError_t err = cudaSuccess;
  auto flags = [&](int *outer, int *inner) {
    if (err == cudaSuccess) err = cudaMemcpyAsync(b->bctl_h, b->bctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (outer) *outer = b->bctl_h->any_outer;
    if (inner) *inner = b->bctl_h->any_inner;
  };
  const cudaGraphConditionalHandle h0 = 0;
  int any_outer = 1;
  while (any_outer && err == cudaSuccess) {
    kb_res<<<Gres, kBlock, 0, st>>>(A.inst, A.tile_inst, A.T, A.Ntot, A.mask, A.qsolve, A.phifx, A.v, A.part, A.c);
    kb_outer<<<n, kBlock, 0, st>>>(A.inst, n, A.T, A.part, A.c, A.bc, A.tol, A.maxit, A.nfam, A.fam_cnt, A.fam_pref,
                                   h0, h0, 0, 0);
    nl += 2;
    flags(&any_outer, nullptr);
    if (!any_outer) break;
    if (vc && err == cudaSuccess) err = cudaGraphLaunch(vc, st), nl += vck;
    kb_cg_b<<<Gb, kBlock, 0, st>>>(A.inst, n, A.pref0, A.T, A.mask, A.vr, A.vu, A.vw, A.part);
    kb_scal<<<n, kBlock, 0, st>>>(A.inst, n, A.T, A.part, A.c, A.bc, A.eta, A.tol_abs, A.maxit, 1, A.nfam, A.fam_cnt,
                                  A.fam_pref, h0, 0);
    nl += 2;
    int any_inner = 0;
    flags(nullptr, &any_inner);
    while (any_inner && err == cudaSuccess) {
      kb_cg_a<<<Ga, kBlock, 0, st>>>(A.inst, n, A.pref0, A.T, A.mask, A.v, A.part, A.c);
      if (vc) err = cudaGraphLaunch(vc, st), nl += vck;
      kb_cg_b<<<Gb, kBlock, 0, st>>>(A.inst, n, A.pref0, A.T, A.mask, A.vr, A.vu, A.vw, A.part);
      kb_scal<<<n, kBlock, 0, st>>>(A.inst, n, A.T, A.part, A.c, A.bc, A.eta, A.tol_abs, A.maxit, 0, A.nfam,
                                    A.fam_cnt, A.fam_pref, h0, 0);
      nl += 3;
      flags(nullptr, &any_inner);
    }
    kb_correct<<<Gcor, kBlock, 0, st>>>(A.inst, A.tile_inst, A.T, A.mask, A.vx, A.phifx, A.phi32, A.flag, A.c);
    nl += 1;
  }
  if (vc) cudaGraphExecDestroy(vc);
  BCK(b, err);
  BCK(b, cudaGetLastError());
  BCK(b, rec(3));
  return LBE_OK;
}

// after a profiled step: accumulate the phase times
int profile_collect(lbe_batch *b) {
  BCK(b, cudaEventSynchronize(b->ev[3]));
  float t[3];
  for (int k = 0; k < 3; ++k) {
    BCK(b, cudaEventElapsedTime(&t[k], b->ev[k], b->ev[k + 1]));
    b->prof_ms[k] += t[k];
  }
  b->prof_steps += 1;
  return LBE_OK;
}

// the FP64 copy of the potential brought up to date (charges, fields)
cudaError_t sync_phi64(lbe_batch *b) {
  if (!b->phi64_stale) return cudaSuccess;
  lbe::kb_phi_to64<<<b->grid > 0 ? b->grid : 1024, lbe::kBlock, 0, b->stream>>>(b->Ntot, b->phifx, b->phi);
  b->phi64_stale = false;
  return cudaGetLastError();
}

// launch one step (or, step = false, one solve): one graph launch, or the
// host-polled sequence
int launch_step(lbe_batch *b, bool step) {
  b->phi64_stale = true;  // the solve (and the warm start) move the fixed-point potential
  const float *fin = b->f[0];
  float *fout = b->f[0];
  if (b->polled) {
    const int rc = run_polled(b, step, fin, fout, b->q, b->qstar);
    if (rc != LBE_OK) return rc;
  } else if (!step) {
    if (!b->exec[4]) BCK(b, build_graph(b, false, nullptr, nullptr, b->q, b->qstar, &b->exec[4]));
    BCK(b, cudaGraphLaunch(b->exec[4], b->stream));
    return LBE_OK;
  } else {
    const int base = b->profiling ? 5 : 0;
    int slot = -1, empty = -1;
    for (int k = base; k < base + 4; ++k) {
      if (b->exec[k] && b->key_odd[k] == (int)b->aa_odd && b->key_q[k] == b->q) slot = k;
      if (!b->exec[k] && empty < 0) empty = k;
    }
    if (slot < 0) {
      if (empty < 0) return bfail(b, LBE_ERR_STATE, "batch: graph cache full");
      BCK(b, build_graph(b, true, fin, fout, b->q, b->qstar, &b->exec[empty], b->profiling));
      b->key_odd[empty] = (int)b->aa_odd;
      b->key_q[empty] = b->q;
      slot = empty;
    }
    BCK(b, cudaGraphLaunch(b->exec[slot], b->stream));
  }
  if (!step) return LBE_OK;
  if (b->flow) {
    b->aa_odd = !b->aa_odd;
  } else {
    int64_t *t = b->q;
    b->q = b->qstar;
    b->qstar = t;
  }
  if (b->profiling) return profile_collect(b);
  return LBE_OK;
}

int read_status(lbe_batch *b) {
  BCK(b, cudaMemcpyAsync(b->bctl_h, b->bctl, sizeof(lbe::BatchCtl), cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  std::vector<lbe::InstCtl> c(b->n);
  BCK(b, cudaMemcpy(c.data(), b->ictl, sizeof(lbe::InstCtl) * b->n, cudaMemcpyDeviceToHost));
  b->stats.poisson_iters = b->bctl_h->total_iters;
  b->stats.poisson_solves = (int)b->bctl_h->solves;
  long long mx = b->bctl_h->max_iters;
  int worst = 0;
  double res = 0.0;
  for (auto &x : c) {
    if (x.status) worst = x.status;
    if (x.res > res) res = x.res;
    if (x.iters > mx) mx = x.iters;
  }
  b->stats.poisson_max_iters = (int)mx;
  if (!worst) worst = b->bctl_h->sticky_status;
  b->stats.poisson_residual = res;
  if (worst == LBE_ERR_NOCONVERGE) return bfail(b, LBE_ERR_NOCONVERGE, "batch poisson: no convergence");
  if (worst == LBE_ERR_NONFINITE) return bfail(b, LBE_ERR_NONFINITE, "batch poisson: non-finite residual");
  return LBE_OK;
}

int flags(lbe_batch *b) {
  int v = 0;
  BCK(b, cudaMemcpy(&v, b->flag, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) return bfail(b, LBE_ERR_NONFINITE, "state out of range: fixed-point solute, solvent density or a NaN");
  return LBE_OK;
}

// Autotuner: the persistent grid is k * SM-count blocks; each candidate k is
// timed on the sweep (the heaviest kernel, on the real instance mix) and the
// fastest kept.  The sweep only writes buffers that the next step rewrites
// (populations out, flux-updated solute, velocity), so tuning leaves the
// state unchanged.
int autotune(lbe_batch *b) {
  using namespace lbe;
  int dev = 0, sms = 0;
  BCK(b, cudaGetDevice(&dev));
  BCK(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  static const int cand[LBE_BATCH_TUNE_CANDIDATES] = {1, 2, 3, 4, 6, 8};
  cudaEvent_t e0, e1;
  BCK(b, cudaEventCreate(&e0));
  BCK(b, cudaEventCreate(&e1));
  float best = 1e30f;
  int best_grid = 4 * sms;
  // the sweep reads the link records of the current state; the trial sweeps
  // update the populations in place, which are put back to rest (the state
  // kb_init left) afterwards
  prep_kernel(b->Ntot)<<<4 * sms, kBlock, 0, b->stream>>>(b->inst_d, b->tile_inst, b->T, (int)b->Ntot, b->phi32,
                                                         b->q, b->lf);
  cudaError_t err = cudaGetLastError();
  for (int c = 0; c < LBE_BATCH_TUNE_CANDIDATES && err == cudaSuccess; ++c) {
    const int grid = cand[c] * sms;
    float ms = 0.f;
    for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
      err = cudaEventRecord(e0, b->stream);
      sweep_kernel(b->flow, b->Ntot, false)<<<grid, kBlock, 0, b->stream>>>(
          b->inst_d, b->tile_inst, b->T, (int)b->Ntot, b->mask, b->f[0], b->f[0], b->q, b->qstar, b->lf, b->u,
          b->flag);
      if (err == cudaSuccess) err = cudaGetLastError();
      if (err == cudaSuccess) err = cudaEventRecord(e1, b->stream);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float t = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0) ms += t;  // the first launch warms up
    }
    b->tuned_ms[c] = ms / 2;
    if (ms < best) {
      best = ms;
      best_grid = grid;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BCK(b, err);
  BCK(b, cudaMemsetAsync(b->f[0], 0, sizeof(float) * lbe::kQ * b->Ntot, b->stream));  // rest: zero deviations
  BCK(b, cudaMemsetAsync(b->u, 0, sizeof(float4) * b->Ntot, b->stream));
  b->aa_odd = false;
  b->grid = best_grid;
  return LBE_OK;
}

}  // namespace

extern "C" {

const char *lbe_batch_last_error(const lbe_batch *b) { return b ? b->err.c_str() : "invalid batch"; }

int lbe_batch_create(const lbe_params *params, int n, void *cuda_stream, lbe_batch **out) {
  if (!params || !out || n < 1) return LBE_ERR_ARG;
  *out = nullptr;
  long long Ntot = 0, T = 0;
  for (int i = 0; i < n; ++i) {
    const lbe_params &p = params[i];
    if (p.precision != LBE_FP32 || p.nspecies != 2 || p.z[0] != 1.0 || p.z[1] != -1.0 ||
        p.rho_bulk[0] != p.rho_bulk[1] || !(p.rho_bulk[0] > 0.0))
      return LBE_ERR_ARG;  // batched form: FP32, 1:1 salt
    if (p.flow != params[0].flow || p.poisson_tol != params[0].poisson_tol ||
        p.poisson_max_iter != params[0].poisson_max_iter)
      return LBE_ERR_ARG;
    if (p.nx < 1 || p.ny < 1 || p.nz < 1 || !(p.tau > 0.5) || !(p.bjerrum > 0.0) || !(p.D[0] >= 0.0) ||
        !(p.D[1] >= 0.0) || !(p.poisson_tol > 0.0) || p.poisson_max_iter < 1)
      return LBE_ERR_ARG;
    const long long N = (long long)p.nx * p.ny * p.nz;
    Ntot += N;
    T += (N + lbe::kTile - 1) / lbe::kTile;
  }
  // 32-bit node indices; component offsets of the 3 velocity components stay
  // below 2^31 (the population components are offset in 64 bits)
  if (3 * Ntot >= (1LL << 31)) return LBE_ERR_ARG;
  lbe_batch *b = new lbe_batch();
  b->n = n;
  b->prm.assign(params, params + n);
  b->flow = params[0].flow != 0;
  b->Ntot = Ntot;
  b->T = (int)T;
  b->ids.resize(n);
  b->psi.assign((size_t)n * (kBE + 1), 0.0);
  b->have_geometry.assign(n, 0);
  b->inst.resize(n);
  // per-instance constants: the single-lattice code derives them
  long long off = 0, t0 = 0;
  std::vector<int> tile_inst((size_t)T);
  for (int i = 0; i < n; ++i) {
    lbe_handle tmp;
    tmp.prm = params[i];
    const lbe_params &p = params[i];
    const long long N = (long long)p.nx * p.ny * p.nz;
    lbe::fill_constants(&tmp);
    lbe::InstDev &I = b->inst[i];
    I.g = lbe::Geo{p.nx, p.ny, p.nz, p.periodic[0] != 0, p.periodic[1] != 0, p.periodic[2] != 0, N};
    I.off = (int)off;
    I.tile0 = (int)t0;
    I.ntiles = (int)((N + lbe::kTile - 1) / lbe::kTile);
    I.fx = lbe::make_fastdiv((uint32_t)p.nx);
    I.fxy = lbe::make_fastdiv((uint32_t)(p.nx * p.ny));
    if (!lbe::fastdiv_ok(I.fx, (uint32_t)N) || !lbe::fastdiv_ok(I.fxy, (uint32_t)N)) {
      delete b;
      return LBE_ERR_ARG;
    }
    I.n_elec = 0;
    I.selfmask = tmp.phys.selfmask;
    I.four_pi_lb = tmp.phys.four_pi_lb;
    {
      const double c6 = 6.0 * tmp.phys.four_pi_lb * tmp.p32.sd[0];
      I.c6_hi = (float)c6;
      I.c6_lo = (float)(c6 - (double)I.c6_hi);
    }
    I.eps = tmp.phys.eps;
    I.P = tmp.p32;
    for (int k = 0; k < I.ntiles; ++k) tile_inst[(size_t)(t0 + k)] = i;
    off += N;
    t0 += I.ntiles;
  }
  const bool own = cuda_stream == nullptr;
  if (own) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return LBE_ERR_CUDA;
    }
  } else {
    b->stream = (cudaStream_t)cuda_stream;
  }
  b->owns_stream = own;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
  };
  const size_t N = (size_t)Ntot;
  alloc((void **)&b->inst_d, sizeof(lbe::InstDev) * n);
  alloc((void **)&b->tile_inst, sizeof(int) * T);
  alloc((void **)&b->id, N);
  alloc((void **)&b->mask, 4 * N);
  alloc((void **)&b->f[0], 4 * N * lbe::kQ);  // one buffer: the populations are updated in place
  alloc((void **)&b->q, 8 * N * 2);
  alloc((void **)&b->qstar, 8 * N * 2);
  alloc((void **)&b->phi, 8 * N);
  alloc((void **)&b->phi_prev, 8 * lbe::kHist * N);
  alloc((void **)&b->phi32, 4 * N);
  alloc((void **)&b->lf, sizeof(float4) * N);
  alloc((void **)&b->phifx, 8 * N);
  alloc((void **)&b->u, sizeof(float4) * N);
  alloc((void **)&b->vec, 4 * N * 6);
  alloc((void **)&b->part, sizeof(double) * 3 * T);
  alloc((void **)&b->psi_d, sizeof(double) * n * (kBE + 1));
  alloc((void **)&b->ictl, sizeof(lbe::InstCtl) * n);
  alloc((void **)&b->bctl, sizeof(lbe::BatchCtl));
  alloc((void **)&b->qpart, sizeof(double) * kBE * T);
  alloc((void **)&b->qout, sizeof(double) * kBE * n);
  alloc((void **)&b->flag, sizeof(int));
  alloc((void **)&b->hist, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->bctl_h, sizeof(lbe::BatchCtl));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->qhost, sizeof(double) * kBE * n);
  if (e == cudaSuccess) e = cudaMemcpy(b->tile_inst, tile_inst.data(), sizeof(int) * T, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->ictl, 0, sizeof(lbe::InstCtl) * n);
  if (e == cudaSuccess) e = cudaMemset(b->bctl, 0, sizeof(lbe::BatchCtl));
  if (e == cudaSuccess) e = cudaMemset(b->flag, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->hist, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->u, 0, sizeof(float4) * N);
  if (e != cudaSuccess) {
    bfree(b);
    if (own) cudaStreamDestroy(b->stream);
    delete b;
    return LBE_ERR_CUDA;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->grid = 4 * (sms > 0 ? sms : 152);
  const char *env = getenv("LBE_POISSON_GRAPH");
  b->polled = env && env[0] == '0';
  *out = b;
  return LBE_OK;
}

int lbe_batch_destroy(lbe_batch *b) {
  if (!b) return LBE_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  bfree(b);
  if (b->owns_stream) cudaStreamDestroy(b->stream);
  delete b;
  return LBE_OK;
}

int lbe_batch_set_geometry(lbe_batch *b, int i, const uint8_t *node_id, int n_electrodes) {
  if (!b) return LBE_ERR_ARG;
  if (i < 0 || i >= b->n || !node_id || n_electrodes < 0 || n_electrodes > kBE)
    return bfail(b, LBE_ERR_ARG, "batch set_geometry: bad arguments");
  const lbe::InstDev &I = b->inst[i];
  const lbe::Geo &g = I.g;
  std::vector<uint8_t> ids(node_id, node_id + g.N);
  for (long long r = 0; r < g.N; ++r) {
    if (ids[r] > n_electrodes) return bfail(b, LBE_ERR_GEOMETRY, "batch set_geometry: id exceeds n_electrodes");
    if (ids[r]) continue;
    int x, y, z;
    lbe::coords(g, r, x, y, z);
    if ((!g.px && (x == 0 || x == g.nx - 1)) || (!g.py && (y == 0 || y == g.ny - 1)) ||
        (!g.pz && (z == 0 || z == g.nz - 1)))
      return bfail(b, LBE_ERR_GEOMETRY, "batch set_geometry: fluid node on a non-periodic face");
  }
  b->ids[i] = std::move(ids);
  b->inst[i].n_elec = n_electrodes;
  b->have_geometry[i] = 1;
  b->initialised = false;
  return LBE_OK;
}

int lbe_batch_set_voltage(lbe_batch *b, int i, const double *psi) {
  if (!b) return LBE_ERR_ARG;
  if (i < 0 || i >= b->n || !psi) return bfail(b, LBE_ERR_ARG, "batch set_voltage: bad arguments");
  if (b->initialised) return bfail(b, LBE_ERR_STATE, "batch set_voltage: set voltages before lbe_batch_init");
  for (int e = 0; e < b->inst[i].n_elec; ++e) {
    if (!isfinite(psi[e])) return bfail(b, LBE_ERR_ARG, "batch set_voltage: non-finite potential");
    if (!(fabs(psi[e]) < lbe::kPhiMax))
      return bfail(b, LBE_ERR_ARG, "batch set_voltage: potentials are held below 100 in magnitude");
    b->psi[(size_t)i * (kBE + 1) + e + 1] = psi[e];
  }
  return LBE_OK;
}

int lbe_batch_init(lbe_batch *b) {
  using namespace lbe;
  if (!b) return LBE_ERR_ARG;
  for (int i = 0; i < b->n; ++i)
    if (!b->have_geometry[i]) return bfail(b, LBE_ERR_STATE, "batch init: an instance has no geometry");
  // geometry: ids, link masks (per instance, set-up only)
  for (int i = 0; i < b->n; ++i) {
    const InstDev &I = b->inst[i];
    BCK(b, cudaMemcpyAsync(b->id + I.off, b->ids[i].data(), I.g.N, cudaMemcpyHostToDevice, b->stream));
    BCK(b, launch_build_mask(I.g, b->id + I.off, b->mask + I.off, b->stream));
  }
  int rc = mg_setup(b);  // also uploads the instance table
  if (rc != LBE_OK) return rc;
  BCK(b, cudaMemcpyAsync(b->psi_d, b->psi.data(), sizeof(double) * b->psi.size(), cudaMemcpyHostToDevice, b->stream));
  b->aa_odd = false;
  kb_init<<<b->grid, kBlock, 0, b->stream>>>(b->inst_d, b->tile_inst, b->T, b->Ntot, b->id, b->psi_d, b->f[0], b->q,
                                             b->phi, b->phi32, b->phifx, b->phi_prev, b->u);
  BCK(b, cudaGetLastError());
  BCK(b, cudaMemsetAsync(b->hist, 0, sizeof(int), b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  drop_graphs(b);
  rc = autotune(b);
  if (rc != LBE_OK) return rc;
  BCK(b, cudaMemsetAsync(b->flag, 0, sizeof(int), b->stream));
  BCK(b, cudaMemsetAsync(b->bctl, 0, sizeof(BatchCtl), b->stream));
  rc = launch_step(b, false);
  if (rc != LBE_OK) return rc;
  rc = read_status(b);
  if (rc == LBE_OK) b->initialised = true;
  return rc;
}

int lbe_batch_step(lbe_batch *b, int nsteps) {
  using namespace lbe;
  if (!b) return LBE_ERR_ARG;
  if (!b->initialised) return bfail(b, LBE_ERR_STATE, "batch step: call lbe_batch_init first");
  if (nsteps < 0) return bfail(b, LBE_ERR_ARG, "batch step: negative step count");
  BCK(b, cudaMemsetAsync(b->bctl, 0, sizeof(BatchCtl), b->stream));
  for (int s = 0; s < nsteps; ++s) {
    const int rc = launch_step(b, true);
    if (rc != LBE_OK) return rc;
  }
  int rc = read_status(b);
  if (b->profiling) {
    b->prof_iters += b->stats.poisson_iters;
    b->prof_solves += b->stats.poisson_solves;
  }
  // a state out of range (range flag) explains a solve that failed after it
  const int frc = flags(b);
  return frc != LBE_OK ? frc : rc;
}

int lbe_batch_charge(lbe_batch *b, double *q_out, int out_on_device) {
  using namespace lbe;
  if (!b) return LBE_ERR_ARG;
  if (!b->initialised) return bfail(b, LBE_ERR_STATE, "batch charge: call lbe_batch_init first");
  if (!q_out) return bfail(b, LBE_ERR_ARG, "batch charge: NULL output");
  BCK(b, sync_phi64(b));
  kb_charge<<<b->grid, kBlock, 0, b->stream>>>(b->inst_d, b->tile_inst, b->T, b->id, b->mask, b->phi, b->qpart);
  kb_charge_final<<<b->n, 32, 0, b->stream>>>(b->inst_d, b->T, b->qpart, b->qout);
  BCK(b, cudaGetLastError());
  const size_t bytes = sizeof(double) * kBE * b->n;
  if (out_on_device) {
    BCK(b, cudaMemcpyAsync(q_out, b->qout, bytes, cudaMemcpyDeviceToDevice, b->stream));
  } else {
    BCK(b, cudaMemcpyAsync(b->qhost, b->qout, bytes, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    memcpy(q_out, b->qhost, bytes);
  }
  return LBE_OK;
}

int lbe_batch_fields(lbe_batch *b, int i, int which, double *out, int out_on_device) {
  using namespace lbe;
  if (!b) return LBE_ERR_ARG;
  if (!b->initialised) return bfail(b, LBE_ERR_STATE, "batch fields: call lbe_batch_init first");
  if (i < 0 || i >= b->n || !out || (which != LBE_FIELD_PHI && which != LBE_FIELD_N))
    return bfail(b, LBE_ERR_ARG, "batch fields: bad arguments (PHI or N)");
  const InstDev &I = b->inst[i];
  const size_t count = (size_t)I.g.N * (which == LBE_FIELD_N ? 2 : 1);
  double *dst = out, *tmp = nullptr;
  if (!out_on_device) {
    BCK(b, cudaMalloc(&tmp, count * sizeof(double)));
    dst = tmp;
  }
  cudaError_t e;
  if (which == LBE_FIELD_PHI) {
    e = sync_phi64(b);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst, b->phi + I.off, sizeof(double) * I.g.N, cudaMemcpyDeviceToDevice, b->stream);
  } else {
    kb_n_to_double<<<(unsigned)((I.g.N + 255) / 256), 256, 0, b->stream>>>(b->inst_d, i, b->Ntot, b->q, b->mask, dst);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !out_on_device) e = cudaMemcpyAsync(out, tmp, count * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (tmp) cudaFree(tmp);
  BCK(b, e);
  return LBE_OK;
}

int lbe_batch_get_stats(const lbe_batch *b, lbe_stats *out) {
  if (!b || !out) return LBE_ERR_ARG;
  *out = b->stats;
  return LBE_OK;
}

int lbe_batch_profile_begin(lbe_batch *b) {
  if (!b) return LBE_ERR_ARG;
  for (int k = 0; k < 4; ++k)
    if (!b->ev[k]) BCK(b, cudaEventCreate(&b->ev[k]));
  b->profiling = true;
  b->prof_ms[0] = b->prof_ms[1] = b->prof_ms[2] = 0.0;
  b->prof_steps = b->prof_iters = b->prof_solves = b->prof_launches = 0;
  return LBE_OK;
}

int lbe_batch_profile_end(lbe_batch *b, lbe_profile *out) {
  if (!b || !out) return LBE_ERR_ARG;
  BCK(b, cudaStreamSynchronize(b->stream));
  memset(out, 0, sizeof(*out));
  out->sweep_ms = b->prof_ms[0];
  out->advect_ms = b->prof_ms[1];
  out->poisson_ms = b->prof_ms[2];
  out->sweep_launches = b->prof_steps;
  out->advect_launches = b->flow ? b->prof_steps : 0;
  out->poisson_solves = b->prof_solves;
  out->poisson_iters = b->prof_iters;
  out->kernel_launches = b->polled ? b->prof_launches : -1;
  b->profiling = false;
  return LBE_OK;
}

int lbe_batch_tuning(const lbe_batch *b, int *grid_blocks, double *ms_out) {
  if (!b) return LBE_ERR_ARG;
  if (grid_blocks) *grid_blocks = b->grid;
  if (ms_out)
    for (int c = 0; c < LBE_BATCH_TUNE_CANDIDATES; ++c) ms_out[c] = b->tuned_ms[c];
  return LBE_OK;
}

}  // extern "C"
