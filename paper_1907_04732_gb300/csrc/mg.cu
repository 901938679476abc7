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
// prolongation+post-smoothing kernels and two on the finest level.
#include <string.h>

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
// shuffle sum of the children's pre-smoothed residuals.  The coarse node's
// residual rc and its pre-smoothed iterate zc = omega rc/diag are stored.
__device__ __forceinline__ void coarse_of_thread(const MgLevel &C, int &I, int &X, int &Y, int &Z, int &ch) {
  const int t = threadIdx.x;
  I = blockIdx.x * (blockDim.x / 8) + (t >> 3);
  ch = t & 7;
  X = Y = Z = 0;
  if (I < C.N) level_coords(C, I, X, Y, Z);
}

__device__ __forceinline__ void store_coarse(const MgLevel &C, int I, float v, const float *__restrict__ AC,
                                             float *__restrict__ rc, float *__restrict__ zc) {
  const float d = AC[13 * C.S + I];
  rc[I] = v;
  zc[I] = d != 0.f ? kOmega * v / d : 0.f;
}

// level 1: a fluid child's pre-smoothed residual is r - omega A u, u = r/diag
// being the Jacobi vector the CG formed
__global__ void __launch_bounds__(256) k_restrict0(const Geo g, uint32_t selfmask, const uint32_t *__restrict__ mask,
                                                   const float *__restrict__ r, const float *__restrict__ u,
                                                   const MgLevel C, const float *__restrict__ AC,
                                                   float *__restrict__ rc, float *__restrict__ zc,
                                                   const PoissonCtl *c) {
  if (c->inner_done) return;
  int I, X, Y, Z, ch, x, y, z;
  coarse_of_thread(C, I, X, Y, Z, ch);
  float v = 0.f;
  if (I < C.N && child_of(C, X, Y, Z, ch, g.nx, g.ny, g.nz, x, y, z)) {
    const int i = x + g.nx * (y + g.ny * z);
    const uint32_t m = mask[i];
    if (m & kFluidBit) {
      const float s6 = nbsum6(m, selfmask, offsets_of(g, x, y, z), i, u);
      v = r[i] - kOmega * ((float)diag6(m, selfmask) * u[i] - s6) * (1.f / 6.f);
    }
  }
  v = sum8(v);
  if (ch == 0 && I < C.N) store_coarse(C, I, v, AC, rc, zc);
}

__global__ void __launch_bounds__(256) k_restrict(const MgLevel F, const float *__restrict__ AF,
                                                  const float *__restrict__ r, const float *__restrict__ zf,
                                                  const MgLevel C, const float *__restrict__ AC,
                                                  float *__restrict__ rc, float *__restrict__ zc,
                                                  const PoissonCtl *c) {
  if (c->inner_done) return;
  int I, X, Y, Z, ch, x, y, z;
  coarse_of_thread(C, I, X, Y, Z, ch);
  float v = 0.f;
  if (I < C.N && child_of(C, X, Y, Z, ch, F.nx, F.ny, F.nz, x, y, z)) v = presmoothed_res_z(F, AF, r, zf, x, y, z);
  v = sum8(v);
  if (ch == 0 && I < C.N) store_coarse(C, I, v, AC, rc, zc);
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
__global__ void k_prolong0(const Geo g, const uint32_t *__restrict__ mask, const float *__restrict__ u,
                           const MgLevel C, const float *__restrict__ ec, float *__restrict__ t,
                           const PoissonCtl *c) {
  if (c->inner_done) return;
  int x, y, z;
  long long il;
  if (!node_of(g, 1, 0, x, y, z, il)) return;
  const int i = (int)il;
  t[i] = (mask[i] & kFluidBit) ? fmaf(kAlpha, ec[agg_index(C, x, y, z)], kOmega * u[i]) : 0.f;
}

__global__ void k_post0(const Geo g, uint32_t selfmask, const uint32_t *__restrict__ mask, const float *__restrict__ r,
                        const float *__restrict__ t, float *__restrict__ u, const PoissonCtl *c) {
  if (c->inner_done) return;
  int x, y, z;
  long long il;
  if (!node_of(g, 1, 0, x, y, z, il)) return;
  const int i = (int)il;
  const uint32_t m = mask[i];
  if (!(m & kFluidBit)) {
    u[i] = 0.f;
    return;
  }
  const float d6 = (float)diag6(m, selfmask);
  const float s6 = nbsum6(m, selfmask, offsets_of(g, x, y, z), i, t);
  const float ti = t[i];
  u[i] = ti + kOmega * __fdividef(6.f * r[i] - (d6 * ti - s6), d6);
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
  return cudaGetLastError();
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
  mg = MGWork{};
}

// u = M r as a sequence of kernels, either launched on the stream or added to
// a graph (gr != nullptr) after *last
cudaError_t mg_vcycle(lbe_handle *h, const float *r0, float *u0, const PoissonCtl *c, cudaGraph_t gr,
                      cudaGraphNode_t *last, cudaStream_t st) {
  MGWork &mg = h->mg;
  const int nl = mg.nlev;
  const Geo g = h->geo;
  const Launch L0 = make_launch(g);
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
  auto cgrid = [](const MgLevel &C) { return dim3((unsigned)((C.N * 8 + 255) / 256)); };
  // down: restrictions (pre-smoothing on the fly)
  nodes.push_back(Node{(void *)k_restrict0, cgrid(lv[1]), dim3(256),
                       {(void *)pg, (void *)psm, P(h->mask), P(r0), P(u0), &lv[1], P(mg.lv[1].A), P(mg.lv[1].r),
                        P(mg.lv[1].z), P(c)}});
  for (int l = 1; l < nl - 1; ++l)
    nodes.push_back(Node{(void *)k_restrict, cgrid(lv[l + 1]), dim3(256),
                         {&lv[l], P(mg.lv[l].A), P(mg.lv[l].r), P(mg.lv[l].z), &lv[l + 1], P(mg.lv[l + 1].A),
                          P(mg.lv[l + 1].r), P(mg.lv[l + 1].z), P(c)}});
  // coarsest
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
                       {(void *)pg, P(h->mask), P(u0), &lv[1], P(mg.lv[1].e), P(mg.t0), P(c)}});
  nodes.push_back(Node{(void *)k_post0, L0.grid, L0.block,
                       {(void *)pg, (void *)psm, P(h->mask), P(r0), P(mg.t0), P(u0), P(c)}});
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
