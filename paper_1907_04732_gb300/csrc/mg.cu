// Geometric multigrid preconditioner of the FP32 Poisson correction solve.
//
// The CG of the Poisson solve (poisson.cu) needs u = M r with M ~ A^-1; the
// plain Jacobi choice M = D^-1 leaves it O(L) iterations on an L-long gap.
// Here M is one symmetric V-cycle; the hierarchy, smoother and correction
// are described with their per-node arithmetic in mg_device.cuh.  Any
// symmetric positive definite M leaves the CG fixed point unchanged.
//
// Kernels per V-cycle: the pre-smoothing sweep from zero (e = omega r/diag)
// is evaluated on the fly where it is needed (restriction, prolongation), so
// a cycle over levels 0..L is L restrictions, the coarsest solve, L-1 fused
// prolongation+post-smoothing kernels and two on the finest level.  The
// coarsest level is solved exactly (its inverse, formed once on the host)
// where its operator is positive definite: a weak coarse solve costs CG
// iterations (on the 64x64x256 electro-osmosis lattice 3.2 per step with 32
// Jacobi sweeps, 2.6 with 64 or 128 sweeps or the exact solve).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mg_device.cuh"

namespace lbe {

namespace {

using namespace mgd;

__device__ __forceinline__ bool lnode(const MgLevel &L, int &x, int &y, int &z, int &r) {
  x = blockIdx.x * blockDim.x + threadIdx.x;
  y = blockIdx.y * blockDim.y + threadIdx.y;
  z = blockIdx.z * blockDim.z + threadIdx.z;
  if (x >= L.nx || y >= L.ny || z >= L.nz) return false;
  r = x + L.nx * (y + L.ny * z);
  return true;
}

// --- set-up: level-0 inverse diagonal, Galerkin coarse operators -------------
// level 1 from the fine lattice (mask-defined operator)
__global__ void k_galerkin0(const Geo g, uint32_t selfmask, const uint32_t *__restrict__ mask, const MgLevel C,
                            float *__restrict__ A) {
  int X, Y, Z, I;
  if (!lnode(C, X, Y, Z, I)) return;
  float a[27];
  galerkin0_row(g, selfmask, mask, C, X, Y, Z, a);
#pragma unroll
  for (int d = 0; d < 27; ++d) A[d * C.S + I] = a[d];
}

// level l+1 from level l (27-point)
__global__ void k_galerkin(const MgLevel F, const float *__restrict__ AF, const MgLevel C, float *__restrict__ A) {
  int X, Y, Z, I;
  if (!lnode(C, X, Y, Z, I)) return;
  float a[27];
  galerkin_row(F, AF, C, X, Y, Z, a);
#pragma unroll
  for (int d = 0; d < 27; ++d) A[d * C.S + I] = a[d];
}

// --- V-cycle kernels ---------------------------------------------------------
// Restriction with 8 threads per coarse node (one per child) and a fixed-order
// shuffle sum of the children's pre-smoothed residuals (store_coarse in
// mg_device.cuh).

// level 1: a fluid child's pre-smoothed residual is r - omega A u, u = r/diag
// being the Jacobi vector the CG formed.  A block covers a tile of 32 coarse
// nodes (2^txl along X, the rest along Y; lanes 8k..8k+7 the children of one
// coarse node, child index = lane % 8 as in child_of) on zpb consecutive
// coarse planes: coordinates come from the block and lane indices, with no
// division, and every lane runs the same iterations (the shuffle sum).
__global__ void __launch_bounds__(256) k_restrict0(const Geo g, uint32_t selfmask, const uint32_t *__restrict__ mask,
                                                   const float *__restrict__ r, const float *__restrict__ u,
                                                   const MgLevel C, const float *__restrict__ AC,
                                                   float *__restrict__ rc, float *__restrict__ zc, int txl, int zpb,
                                                   const PoissonCtl *c) {
  if (c->inner_done) return;
  const int ch = threadIdx.x & 7, j = threadIdx.x >> 3;
  const int X = (blockIdx.x << txl) + (j & ((1 << txl) - 1));
  const int Y = blockIdx.y * (32 >> txl) + (j >> txl);
  for (int kz = 0; kz < zpb; ++kz) {
    const int Z = blockIdx.z * zpb + kz;
    const bool own = X < C.nx && Y < C.ny && Z < C.nz;
    int x, y, z;
    float v = 0.f;
    if (own && child_of(C, X, Y, Z, ch, g.nx, g.ny, g.nz, x, y, z)) {
      const int i = x + g.nx * (y + g.ny * z);
      const uint32_t m = mask[i];
      if (m & kFluidBit) {
        const float s6 = nbsum6(m, selfmask, offsets_of(g, x, y, z), i, u);
        v = r[i] - kOmega * ((float)diag6(m, selfmask) * u[i] - s6) * (1.f / 6.f);
      }
    }
    v = sum8(v);
    if (ch == 0 && own) store_coarse(C, X + C.nx * (Y + C.ny * Z), v, AC, rc, zc);
  }
}

__global__ void __launch_bounds__(256) k_restrict(const MgLevel F, const float *__restrict__ AF,
                                                  const float *__restrict__ r, const float *__restrict__ zf,
                                                  const MgLevel C, const float *__restrict__ AC,
                                                  float *__restrict__ rc, float *__restrict__ zc, int txl,
                                                  const PoissonCtl *c) {
  if (c->inner_done) return;
  // the tile mapping of k_restrict0, one coarse plane per block
  const int ch = threadIdx.x & 7, j = threadIdx.x >> 3;
  const int X = (blockIdx.x << txl) + (j & ((1 << txl) - 1));
  const int Y = blockIdx.y * (32 >> txl) + (j >> txl), Z = blockIdx.z;
  const bool own = X < C.nx && Y < C.ny;
  int x, y, z;
  float v = 0.f;
  if (own && child_of(C, X, Y, Z, ch, F.nx, F.ny, F.nz, x, y, z)) v = presmoothed_res_z(F, AF, r, zf, x, y, z);
  v = sum8(v);
  if (ch == 0 && own) store_coarse(C, X + C.nx * (Y + C.ny * Z), v, AC, rc, zc);
}

// fused prolongation + post-smoothing on a 27-point level
__global__ void k_post(const MgLevel L, const float *__restrict__ A, const float *__restrict__ r,
                       const float *__restrict__ z, const MgLevel C, const float *__restrict__ ec,
                       float *__restrict__ out, const PoissonCtl *c) {
  if (c->inner_done) return;
  int X, Y, Z, I;
  if (!lnode(L, X, Y, Z, I)) return;
  out[I] = post_value_z(L, A, r, z, C, ec, X, Y, Z);
}

// level 0: t = omega u + alpha P e_1 (fluid nodes), then
// u = t + omega (r - A t)/diag
__global__ void k_prolong0(const Geo g, int zpt, const uint32_t *__restrict__ mask, const float *__restrict__ u,
                           const MgLevel C, const float *__restrict__ ec, float *__restrict__ t,
                           const PoissonCtl *c) {
  if (c->inner_done) return;
  for (int kz = 0; kz < zpt; ++kz) {
    int x, y, z;
    long long il;
    if (!node_of(g, zpt, kz, x, y, z, il)) continue;
    const int i = (int)il;
    t[i] = (mask[i] & kFluidBit) ? fmaf(kAlpha, ec[agg_index(C, x, y, z)], kOmega * u[i]) : 0.f;
  }
}

__global__ void k_post0(const Geo g, int zpt, uint32_t selfmask, const uint32_t *__restrict__ mask,
                        const float *__restrict__ r, const float *__restrict__ t, float *__restrict__ u,
                        const PoissonCtl *c) {
  if (c->inner_done) return;
  for (int kz = 0; kz < zpt; ++kz) {
    int x, y, z;
    long long il;
    if (!node_of(g, zpt, kz, x, y, z, il)) continue;
    const int i = (int)il;
    const uint32_t m = mask[i];
    if (!(m & kFluidBit)) {
      u[i] = 0.f;
      continue;
    }
    const float d6 = (float)diag6(m, selfmask);
    const float s6 = nbsum6(m, selfmask, offsets_of(g, x, y, z), i, t);
    const float ti = t[i];
    u[i] = ti + kOmega * __fdividef(6.f * r[i] - (d6 * ti - s6), d6);
  }
}

// coarsest level solved exactly: e = A^-1 r with the inverse formed at
// set-up, one warp per row (a fixed summation order)
__global__ void __launch_bounds__(256) k_coarse_direct(int N, const float *__restrict__ Ainv,
                                                       const float *__restrict__ r, float *__restrict__ e,
                                                       const PoissonCtl *c) {
  if (c->inner_done) return;
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= N) return;
  const float *a = Ainv + (size_t)row * N;
  float s = 0.f;
  for (int j = lane; j < N; j += 32) s = fmaf(a[j], r[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) e[row] = s;
}

// coarsest level in one block
__global__ void __launch_bounds__(kCoarseMax) k_coarsest(const MgLevel L, const float *__restrict__ A,
                                                         const float *__restrict__ r, float *__restrict__ e,
                                                         const PoissonCtl *c) {
  if (c->inner_done) return;
  __shared__ float buf[2][kCoarseMax];
  coarsest_solve(L, A, r, e, buf);
}

dim3 lgrid(const MgLevel &L, dim3 &block) {
  const Geo g{L.nx, L.ny, L.nz, 0, 0, 0, L.N};
  const Launch la = make_launch(g);
  block = la.block;
  return la.grid;
}

MgLevel level_dev(const MGLevel &L) { return MgLevel{L.nx, L.ny, L.nz, L.sx, L.sy, L.sz, (int)L.N, L.N}; }


}  // namespace

// build the hierarchy for the current geometry (after the link mask)
// Inverse of the coarsest level's operator from its 27-point rows (host,
// FP64): the operator restricted to the nodes with a non-zero diagonal
// (aggregates holding fluid) is assembled densely, factored A = L L^T
// (Cholesky) and inverted; rows and columns of the other nodes are zero,
// as the Jacobi sweeps leave them.  False when the operator is not
// symmetric positive definite to working accuracy (e.g. a periodic lattice
// without electrodes, whose operator is singular): the sweeps are used then.
bool mgd::coarse_inverse(const MgLevel &L, const std::vector<float> &A27, std::vector<float> &inv) {
  const int N = L.N;
  std::vector<int> act;  // active node -> level index
  std::vector<int> pos(N, -1);
  for (int i = 0; i < N; ++i)
    if (A27[13 * (size_t)N + i] != 0.f) {
      pos[i] = (int)act.size();
      act.push_back(i);
    }
  const int n = (int)act.size();
  inv.assign((size_t)N * N, 0.f);
  if (n == 0) return true;
  std::vector<double> M((size_t)n * n, 0.0);
  for (int a = 0; a < n; ++a) {
    const int I = act[a];
    const int X = I % L.nx, Y = (I / L.nx) % L.ny, Z = I / (L.nx * L.ny);
    for (int q = 0; q < 27; ++q) {
      const float v = A27[(size_t)q * N + I];
      if (v == 0.f) continue;
      auto wr = [](int c, int m) { return c < 0 ? c + m : (c >= m ? c - m : c); };
      const int J = wr(X + q % 3 - 1, L.nx) + L.nx * (wr(Y + (q / 3) % 3 - 1, L.ny) + L.ny * wr(Z + q / 9 - 1, L.nz));
      if (pos[J] < 0) continue;  // a zero of the correction
      M[(size_t)a * n + pos[J]] += (double)v;
    }
  }
  double dmax = 0.0, asym = 0.0, amax = 0.0;
  for (int a = 0; a < n; ++a) {
    dmax = std::max(dmax, M[(size_t)a * n + a]);
    for (int b = 0; b < n; ++b) {
      amax = std::max(amax, std::fabs(M[(size_t)a * n + b]));
      asym = std::max(asym, std::fabs(M[(size_t)a * n + b] - M[(size_t)b * n + a]));
    }
  }
  if (!(dmax > 0.0) || asym > 1e-5 * amax) return false;
  // Cholesky, lower triangle in place
  for (int j = 0; j < n; ++j) {
    double d = M[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= M[(size_t)j * n + k] * M[(size_t)j * n + k];
    if (!(d > 1e-10 * dmax)) return false;
    const double ljj = std::sqrt(d);
    M[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = M[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= M[(size_t)i * n + k] * M[(size_t)j * n + k];
      M[(size_t)i * n + j] = s / ljj;
    }
  }
  // columns of A^-1: solve L y = e_c, L^T x = y
  std::vector<double> x(n);
  for (int cidx = 0; cidx < n; ++cidx) {
    for (int i = 0; i < cidx; ++i) x[i] = 0.0;  // y vanishes above the unit entry
    for (int i = cidx; i < n; ++i) {
      double s = i == cidx ? 1.0 : 0.0;
      for (int k = cidx; k < i; ++k) s -= M[(size_t)i * n + k] * x[k];
      x[i] = s / M[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = x[i];
      for (int k = i + 1; k < n; ++k) s -= M[(size_t)k * n + i] * x[k];
      x[i] = s / M[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) inv[(size_t)act[i] * N + act[cidx]] = (float)x[i];
  }
  return true;
}

cudaError_t mg_setup(lbe_handle *h) {
  MGWork &mg = h->mg;
  mg_free(h);
  const Geo &g = h->geo;
  MgLevel shp[kMaxLevels];
  mg.nlev = level_shapes(g.nx, g.ny, g.nz, shp);
  if (mg.nlev == 0) return cudaSuccess;  // plain Jacobi preconditioning
  for (int l = 1; l < mg.nlev; ++l) {
    MGLevel &L = mg.lv[l];
    L.nx = shp[l].nx;
    L.ny = shp[l].ny;
    L.nz = shp[l].nz;
    L.sx = shp[l].sx;
    L.sy = shp[l].sy;
    L.sz = shp[l].sz;
    L.N = shp[l].N;
  }
  cudaError_t e = cudaMalloc(&mg.t0, sizeof(float) * g.N);
  for (int l = 1; l < mg.nlev && e == cudaSuccess; ++l) {
    MGLevel &L = mg.lv[l];
    e = cudaMalloc(&L.A, sizeof(float) * 27 * L.N);
    if (e == cudaSuccess) e = cudaMalloc(&L.r, sizeof(float) * L.N);
    if (e == cudaSuccess) e = cudaMalloc(&L.e, sizeof(float) * L.N);
    if (e == cudaSuccess) e = cudaMalloc(&L.z, sizeof(float) * L.N);
  }
  if (e != cudaSuccess) {
    mg_free(h);
    return e;
  }
  for (int l = 1; l < mg.nlev; ++l) {
    const MgLevel C = level_dev(mg.lv[l]);
    dim3 blk;
    const dim3 grd = lgrid(C, blk);
    if (l == 1)
      k_galerkin0<<<grd, blk, 0, h->stream>>>(g, h->phys.selfmask, h->mask, C, mg.lv[1].A);
    else
      k_galerkin<<<grd, blk, 0, h->stream>>>(level_dev(mg.lv[l - 1]), mg.lv[l - 1].A, C, mg.lv[l].A);
  }
  cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) return le;
  // the coarsest level is solved exactly where its operator is SPD
  // (LBE_MG_DIRECT=0: Jacobi sweeps everywhere)
  const char *denv = getenv("LBE_MG_DIRECT");
  if (!(denv && denv[0] == '0')) {
    const MGLevel &Lc = mg.lv[mg.nlev - 1];
    std::vector<float> a27((size_t)27 * Lc.N), inv;
    le = cudaMemcpyAsync(a27.data(), Lc.A, sizeof(float) * a27.size(), cudaMemcpyDeviceToHost, h->stream);
    if (le == cudaSuccess) le = cudaStreamSynchronize(h->stream);
    if (le != cudaSuccess) return le;
    if (coarse_inverse(level_dev(Lc), a27, inv)) {
      le = cudaMalloc(&mg.cinv, sizeof(float) * inv.size());
      if (le == cudaSuccess)
        le = cudaMemcpyAsync(mg.cinv, inv.data(), sizeof(float) * inv.size(), cudaMemcpyHostToDevice, h->stream);
      if (le == cudaSuccess) le = cudaStreamSynchronize(h->stream);  // inv is released on return
      if (le != cudaSuccess) return le;
    }
  }
  return cudaSuccess;
}

void mg_free(lbe_handle *h) {
  MGWork &mg = h->mg;
  for (int l = 0; l < kMaxLevels; ++l) {
    cudaFree(mg.lv[l].A);
    cudaFree(mg.lv[l].r);
    cudaFree(mg.lv[l].e);
    cudaFree(mg.lv[l].t);
    cudaFree(mg.lv[l].z);
  }
  cudaFree(mg.t0);
  cudaFree(mg.cinv);
  mg = MGWork{};
}

// u = M r as a sequence of kernels, either launched on the stream or added to
// a graph (gr != nullptr) after *last
cudaError_t mg_vcycle(lbe_handle *h, const float *r0, float *u0, const PoissonCtl *c, cudaGraph_t gr,
                      cudaGraphNode_t *last, cudaStream_t st) {
  MGWork &mg = h->mg;
  const int nl = mg.nlev;
  const Geo g = h->geo;
  // finest-level kernels: the solve's launch (zpt nodes along z per thread)
  const Launch L0 = h->pw.L;
  int zpt0 = L0.zpt;
  const uint32_t sm = h->phys.selfmask;
  // kernel arguments live in these arrays until the nodes are created or the
  // kernels launched
  struct Node {
    void *f;
    dim3 grid, block;
    void *args[12];
  };
  std::vector<Node> nodes;
  std::vector<MgLevel> lv(kMaxLevels);
  std::vector<const void *> ptr;
  ptr.reserve(512);  // no reallocation: the kernel arguments point into it
  auto P = [&](const void *v) -> void * {
    ptr.push_back(v);
    return &ptr.back();
  };
  for (int l = 1; l < nl; ++l) lv[l] = level_dev(mg.lv[l]);
  const void *pg = &g, *psm = &sm;
  // down: restrictions (pre-smoothing on the fly)
  // restrictions: tiles of 32 coarse nodes per block, 2^txl along X (at
  // most 32) and the rest along Y; level 1 with zpb coarse planes per block
  // (at most kSolveBlocks blocks), the others one plane per block
  int txl[kMaxLevels];
  dim3 rgrid[kMaxLevels];
  for (int l = 1; l < nl; ++l) {
    txl[l] = 0;
    while ((1 << txl[l]) < mg.lv[l].nx && txl[l] < 5) ++txl[l];
    rgrid[l] = dim3((unsigned)((mg.lv[l].nx + (1 << txl[l]) - 1) >> txl[l]),
                    (unsigned)((mg.lv[l].ny + (32 >> txl[l]) - 1) / (32 >> txl[l])), (unsigned)mg.lv[l].nz);
  }
  int zpb = (int)(((long long)rgrid[1].x * rgrid[1].y * mg.lv[1].nz + kSolveBlocks - 1) / kSolveBlocks);
  rgrid[1].z = (unsigned)((mg.lv[1].nz + zpb - 1) / zpb);
  nodes.push_back(Node{(void *)k_restrict0, rgrid[1], dim3(256),
                       {(void *)pg, (void *)psm, P(h->mask), P(r0), P(u0), &lv[1], P(mg.lv[1].A), P(mg.lv[1].r),
                        P(mg.lv[1].z), &txl[1], &zpb, P(c)}});
  for (int l = 1; l < nl - 1; ++l)
    nodes.push_back(Node{(void *)k_restrict, rgrid[l + 1], dim3(256),
                         {&lv[l], P(mg.lv[l].A), P(mg.lv[l].r), P(mg.lv[l].z), &lv[l + 1], P(mg.lv[l + 1].A),
                          P(mg.lv[l + 1].r), P(mg.lv[l + 1].z), &txl[l + 1], P(c)}});
  // coarsest: exact (inverse) or Jacobi sweeps
  int ncoarse = (int)mg.lv[nl - 1].N;
  if (mg.cinv)
    nodes.push_back(Node{(void *)k_coarse_direct, dim3((unsigned)((ncoarse + 7) / 8)), dim3(256),
                         {&ncoarse, P(mg.cinv), P(mg.lv[nl - 1].r), P(mg.lv[nl - 1].e), P(c)}});
  else
    nodes.push_back(Node{(void *)k_coarsest, dim3(1), dim3(kCoarseMax),
                         {&lv[nl - 1], P(mg.lv[nl - 1].A), P(mg.lv[nl - 1].r), P(mg.lv[nl - 1].e), P(c)}});
  // up: fused prolongation + post-smoothing on the coarse levels
  for (int l = nl - 2; l >= 1; --l) {
    dim3 blk;
    const dim3 grd = lgrid(lv[l], blk);
    nodes.push_back(Node{(void *)k_post, grd, blk,
                         {&lv[l], P(mg.lv[l].A), P(mg.lv[l].r), P(mg.lv[l].z), &lv[l + 1], P(mg.lv[l + 1].e),
                          P(mg.lv[l].e), P(c)}});
  }
  // finest level
  nodes.push_back(Node{(void *)k_prolong0, L0.grid, L0.block,
                       {(void *)pg, &zpt0, P(h->mask), P(u0), &lv[1], P(mg.lv[1].e), P(mg.t0), P(c)}});
  nodes.push_back(Node{(void *)k_post0, L0.grid, L0.block,
                       {(void *)pg, &zpt0, (void *)psm, P(h->mask), P(r0), P(mg.t0), P(u0), P(c)}});
  cudaError_t e = cudaSuccess;
  for (Node &n : nodes) {
    if (gr) {
      cudaKernelNodeParams kp;
      memset(&kp, 0, sizeof(kp));
      kp.func = n.f;
      kp.gridDim = n.grid;
      kp.blockDim = n.block;
      kp.kernelParams = n.args;
      cudaGraphNode_t nd;
      e = cudaGraphAddKernelNode(&nd, gr, *last ? last : nullptr, *last ? 1 : 0, &kp);
      if (e != cudaSuccess) return e;
      *last = nd;
    } else {
      e = cudaLaunchKernel(n.f, n.grid, n.block, n.args, 0, st);
      if (e != cudaSuccess) return e;
      h->launches += 1;
    }
  }
  return e;
}

// kernels of one V-cycle (launch accounting of the graph path)
int mg_kernels_per_cycle(const lbe_handle *h) { return h->mg.nlev >= 2 ? 2 * (h->mg.nlev - 1) + 2 : 0; }

}  // namespace lbe
