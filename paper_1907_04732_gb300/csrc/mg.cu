// Geometric multigrid preconditioner of the FP32 Poisson correction solve.
//
// The CG of the Poisson solve (poisson.cu) needs u = M r with M ~ A^-1; the
// plain Jacobi choice M = D^-1 leaves it O(L) iterations on an L-long gap.
// Here M is one symmetric V-cycle:
//
//   hierarchy   level 0 is the lattice with the modified-Laplacian operator
//               of Eq. DiscreteLaplacianModif on fluid nodes; level l+1
//               aggregates 2x2x2 nodes of level l (an axis is halved while it
//               is even or non-periodic) and carries the Galerkin operator
//               A_{l+1} = P^T A_l P of the piecewise-constant prolongation P
//               (27-point, built on the GPU; exact for any electrode shape,
//               solid nodes being Dirichlet zeros of the correction)
//   smoother    weighted Jacobi, one sweep before and one after the coarse
//               correction (the same on both sides, so M is symmetric)
//   correction  e += alpha P e_c, alpha > 1 compensating the stiffness of
//               piecewise-constant coarse spaces
//   coarsest    a fixed number of Jacobi sweeps in one thread block
//
// Any symmetric positive definite M leaves the CG fixed point unchanged.
//
// Kernels per V-cycle: the pre-smoothing sweep from zero (e = omega r/diag)
// is evaluated on the fly where it is needed (restriction, prolongation), so
// a cycle over levels 0..L is L restrictions, the coarsest solve, L-1 fused
// prolongation+post-smoothing kernels and two on the finest level.
#include <string.h>

#include "lbe_internal.cuh"

namespace lbe {

namespace {

constexpr float kOmega = 0.7f;     // Jacobi weight
constexpr float kAlpha = 1.6f;     // coarse-correction scaling
constexpr int kCoarseSweeps = 32;  // Jacobi sweeps on the coarsest level
constexpr int kCoarseTarget = 256; // coarsening stops at or below this size
constexpr int kCoarseMax = 1024;   // the coarsest solve owns one node per thread

__host__ __device__ constexpr int d27(int dx, int dy, int dz) { return (dx + 1) + 3 * ((dy + 1) + 3 * (dz + 1)); }

struct LevelDev {
  int nx, ny, nz, px, py, pz;
  int sx, sy, sz;  // 1 when this level halves the axis of the finer level
  int N;
};

__device__ __forceinline__ bool lnode(const LevelDev &L, int &x, int &y, int &z, int &r) {
  x = blockIdx.x * blockDim.x + threadIdx.x;
  y = blockIdx.y * blockDim.y + threadIdx.y;
  z = blockIdx.z * blockDim.z + threadIdx.z;
  if (x >= L.nx || y >= L.ny || z >= L.nz) return false;
  r = x + L.nx * (y + L.ny * z);
  return true;
}

// wrapped coordinate (periodic axes; coordinates stay in range otherwise)
__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// offset of the (coarse) node J relative to I along one axis, in {-1,0,1}
__device__ __forceinline__ int rel(int J, int I, int n) {
  int d = J - I;
  if (d > 1) d -= n;
  if (d < -1) d += n;
  if (n == 2 && d == -1) d = 1;  // on a 2-node periodic axis +1 and -1 coincide
  return d;
}

__device__ __forceinline__ int agg_index(const LevelDev &C, int x, int y, int z) {
  return (x >> C.sx) + C.nx * ((y >> C.sy) + C.ny * (z >> C.sz));
}

// --- set-up: level-0 inverse diagonal, Galerkin coarse operators -------------
__global__ void k_invdiag0(const Geo g, uint32_t selfmask, const uint32_t *__restrict__ mask, float *__restrict__ inv) {
  int x, y, z;
  long long il;
  if (!node_of(g, 1, 0, x, y, z, il)) return;
  const uint32_t m = mask[il];
  if (!(m & kFluidBit)) {
    inv[il] = 0.f;
    return;
  }
  float dg = 0.f;
#pragma unroll
  for (int l = 1; l < kQ; ++l) {
    const uint32_t b = 1u << (l - 1);
    if (selfmask & b) continue;
    dg += (m & b) ? (float)lapc_of(l) : 2.f * (float)lapc_of(l);
  }
  inv[il] = 1.f / dg;
}

// level 1 from the fine lattice (mask-defined operator)
__global__ void k_galerkin0(const Geo g, uint32_t selfmask, const uint32_t *__restrict__ mask, const LevelDev C,
                            float *__restrict__ A) {
  int X, Y, Z, I;
  if (!lnode(C, X, Y, Z, I)) return;
  float a[27];
#pragma unroll
  for (int d = 0; d < 27; ++d) a[d] = 0.f;
  for (int c = 0; c < 8; ++c) {
    const int ax = c & 1, ay = (c >> 1) & 1, az = c >> 2;
    if ((ax && !C.sx) || (ay && !C.sy) || (az && !C.sz)) continue;
    const int x = (X << C.sx) + ax, y = (Y << C.sy) + ay, z = (Z << C.sz) + az;
    if (x >= g.nx || y >= g.ny || z >= g.nz) continue;
    const int i = x + g.nx * (y + g.ny * z);
    const uint32_t m = mask[i];
    if (!(m & kFluidBit)) continue;
    float diag = 0.f;
    for (int l = 1; l < kQ; ++l) {
      const uint32_t b = 1u << (l - 1);
      if (selfmask & b) continue;
      const float w = (float)lapc_of(l);
      if (!(m & b)) {  // link to solid: doubled, Dirichlet
        diag += 2.f * w;
        continue;
      }
      diag += w;
      const int jx = wrap(x + cx_of(l), g.nx), jy = wrap(y + cy_of(l), g.ny), jz = wrap(z + cz_of(l), g.nz);
      const int dx = rel(jx >> C.sx, X, C.nx), dy = rel(jy >> C.sy, Y, C.ny), dz = rel(jz >> C.sz, Z, C.nz);
      a[d27(dx, dy, dz)] -= w;
    }
    a[13] += diag;
  }
#pragma unroll
  for (int d = 0; d < 27; ++d) A[(long long)d * C.N + I] = a[d];
}

// level l+1 from level l (27-point)
__global__ void k_galerkin(const LevelDev F, const float *__restrict__ AF, const LevelDev C, float *__restrict__ A) {
  int X, Y, Z, I;
  if (!lnode(C, X, Y, Z, I)) return;
  float a[27];
#pragma unroll
  for (int d = 0; d < 27; ++d) a[d] = 0.f;
  for (int c = 0; c < 8; ++c) {
    const int ax = c & 1, ay = (c >> 1) & 1, az = c >> 2;
    if ((ax && !C.sx) || (ay && !C.sy) || (az && !C.sz)) continue;
    const int x = (X << C.sx) + ax, y = (Y << C.sy) + ay, z = (Z << C.sz) + az;
    if (x >= F.nx || y >= F.ny || z >= F.nz) continue;
    const int i = x + F.nx * (y + F.ny * z);
    if (AF[13LL * F.N + i] == 0.f) continue;  // inactive node
    for (int d = 0; d < 27; ++d) {
      const float v = AF[(long long)d * F.N + i];
      if (v == 0.f) continue;
      const int jx = wrap(x + d % 3 - 1, F.nx), jy = wrap(y + (d / 3) % 3 - 1, F.ny), jz = wrap(z + d / 9 - 1, F.nz);
      const int dx = rel(jx >> C.sx, X, C.nx), dy = rel(jy >> C.sy, Y, C.ny), dz = rel(jz >> C.sz, Z, C.nz);
      a[d27(dx, dy, dz)] += v;
    }
  }
#pragma unroll
  for (int d = 0; d < 27; ++d) A[(long long)d * C.N + I] = a[d];
}

// --- V-cycle kernels ---------------------------------------------------------
// Restriction with 8 threads per coarse node (one per child) and a fixed-order
// shuffle sum.  The child's residual is r - A e with e = omega r/diag, the
// pre-smoothing sweep from zero, evaluated on the fly.
__device__ __forceinline__ void coarse_of_thread(const LevelDev &C, int &I, int &X, int &Y, int &Z, int &ch) {
  const int t = threadIdx.x;
  I = blockIdx.x * (blockDim.x / 8) + (t >> 3);
  ch = t & 7;
  X = Y = Z = 0;
  if (I < C.N) {
    X = I % C.nx;
    Y = (I / C.nx) % C.ny;
    Z = I / (C.nx * C.ny);
  }
}

__device__ __forceinline__ float sum8(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  return v;
}

__global__ void __launch_bounds__(256) k_restrict0(const Geo g, uint32_t selfmask, const uint32_t *__restrict__ mask,
                                                   const float *__restrict__ r, const float *__restrict__ inv,
                                                   const LevelDev C, float *__restrict__ rc, const PoissonCtl *c) {
  if (c->inner_done) return;
  int I, X, Y, Z, ch;
  coarse_of_thread(C, I, X, Y, Z, ch);
  float v = 0.f;
  const int ax = ch & 1, ay = (ch >> 1) & 1, az = ch >> 2;
  const int x = (X << C.sx) + ax, y = (Y << C.sy) + ay, z = (Z << C.sz) + az;
  if (I < C.N && !((ax && !C.sx) || (ay && !C.sy) || (az && !C.sz)) && x < g.nx && y < g.ny && z < g.nz) {
    const int i = x + g.nx * (y + g.ny * z);
    const uint32_t m = mask[i];
    if (m & kFluidBit) {
      const Offs o = offsets_of(g, x, y, z);
      float s = 0.f, dg = 0.f;
#pragma unroll
      for (int l = 1; l < kQ; ++l) {
        const uint32_t b = 1u << (l - 1);
        if (selfmask & b) continue;
        const float w = (float)lapc_of(l);
        if (m & b) {
          dg += w;
          const int j = i + o.at(cx_of(l), cy_of(l), cz_of(l));
          s += w * (kOmega * r[j] * inv[j]);
        } else {
          dg += 2.f * w;
        }
      }
      const float ri = r[i];
      v = ri - (dg * (kOmega * ri * inv[i]) - s);
    }
  }
  v = sum8(v);
  if (ch == 0 && I < C.N) rc[I] = v;
}

// (A e)(I) on a 27-point level for e = omega r/diag (pre-smoothing from zero)
__device__ __forceinline__ float apply27_first(const LevelDev &L, const float *__restrict__ A,
                                               const float *__restrict__ r, int X, int Y, int Z, int I) {
  float s = 0.f;
#pragma unroll
  for (int d = 0; d < 27; ++d) {
    const float a = A[(long long)d * L.N + I];
    if (a == 0.f) continue;
    const int jx = wrap(X + d % 3 - 1, L.nx), jy = wrap(Y + (d / 3) % 3 - 1, L.ny), jz = wrap(Z + d / 9 - 1, L.nz);
    const int j = jx + L.nx * (jy + L.ny * jz);
    s += a * (kOmega * r[j] / A[13LL * L.N + j]);
  }
  return s;
}

__global__ void __launch_bounds__(256) k_restrict(const LevelDev F, const float *__restrict__ AF,
                                                  const float *__restrict__ r, const LevelDev C,
                                                  float *__restrict__ rc, const PoissonCtl *c) {
  if (c->inner_done) return;
  int I, X, Y, Z, ch;
  coarse_of_thread(C, I, X, Y, Z, ch);
  float v = 0.f;
  const int ax = ch & 1, ay = (ch >> 1) & 1, az = ch >> 2;
  const int x = (X << C.sx) + ax, y = (Y << C.sy) + ay, z = (Z << C.sz) + az;
  if (I < C.N && !((ax && !C.sx) || (ay && !C.sy) || (az && !C.sz)) && x < F.nx && y < F.ny && z < F.nz) {
    const int i = x + F.nx * (y + F.ny * z);
    if (AF[13LL * F.N + i] != 0.f) v = r[i] - apply27_first(F, AF, r, x, y, z, i);
  }
  v = sum8(v);
  if (ch == 0 && I < C.N) rc[I] = v;
}

// corrected iterate of a 27-point level at node j: e = omega r/diag + alpha e_c
__device__ __forceinline__ float corrected(const LevelDev &L, const float *__restrict__ A, const float *__restrict__ r,
                                           const LevelDev &C, const float *__restrict__ ec, int x, int y, int z,
                                           int j) {
  const float d = A[13LL * L.N + j];
  return d != 0.f ? kOmega * r[j] / d + kAlpha * ec[agg_index(C, x, y, z)] : 0.f;
}

// fused prolongation + post-smoothing on a 27-point level:
// out = e + omega (r - A e)/diag with e as in corrected()
__global__ void k_post(const LevelDev L, const float *__restrict__ A, const float *__restrict__ r, const LevelDev C,
                       const float *__restrict__ ec, float *__restrict__ out, const PoissonCtl *c) {
  if (c->inner_done) return;
  int X, Y, Z, I;
  if (!lnode(L, X, Y, Z, I)) return;
  const float d = A[13LL * L.N + I];
  if (d == 0.f) {
    out[I] = 0.f;
    return;
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const float a = A[(long long)q * L.N + I];
    if (a == 0.f) continue;
    const int jx = wrap(X + q % 3 - 1, L.nx), jy = wrap(Y + (q / 3) % 3 - 1, L.ny), jz = wrap(Z + q / 9 - 1, L.nz);
    s += a * corrected(L, A, r, C, ec, jx, jy, jz, jx + L.nx * (jy + L.ny * jz));
  }
  const float e = corrected(L, A, r, C, ec, X, Y, Z, I);
  out[I] = e + kOmega * (r[I] - s) / d;
}

// level 0: t = omega r/diag + alpha P e_1 (fluid nodes), then
// u = t + omega (r - A t)/diag
__global__ void k_prolong0(const Geo g, const uint32_t *__restrict__ mask, const float *__restrict__ r,
                           const float *__restrict__ inv, const LevelDev C, const float *__restrict__ ec,
                           float *__restrict__ t, const PoissonCtl *c) {
  if (c->inner_done) return;
  int x, y, z;
  long long il;
  if (!node_of(g, 1, 0, x, y, z, il)) return;
  const int i = (int)il;
  t[i] = (mask[i] & kFluidBit) ? kOmega * r[i] * inv[i] + kAlpha * ec[agg_index(C, x, y, z)] : 0.f;
}

__global__ void k_post0(const Geo g, uint32_t selfmask, const uint32_t *__restrict__ mask, const float *__restrict__ r,
                        const float *__restrict__ inv, const float *__restrict__ t, float *__restrict__ u,
                        const PoissonCtl *c) {
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
  const Offs o = offsets_of(g, x, y, z);
  float s = 0.f, dg = 0.f;
#pragma unroll
  for (int l = 1; l < kQ; ++l) {
    const uint32_t b = 1u << (l - 1);
    if (selfmask & b) continue;
    const float w = (float)lapc_of(l);
    if (m & b) {
      dg += w;
      s += w * t[i + o.at(cx_of(l), cy_of(l), cz_of(l))];
    } else {
      dg += 2.f * w;
    }
  }
  const float ti = t[i];
  u[i] = ti + kOmega * (r[i] - (dg * ti - s)) * inv[i];
}

// coarsest level: kCoarseSweeps weighted Jacobi sweeps from zero in one
// block, one node per thread, iterates in shared memory
__global__ void __launch_bounds__(kCoarseMax) k_coarsest(const LevelDev L, const float *__restrict__ A,
                                                         const float *__restrict__ r, float *__restrict__ e,
                                                         const PoissonCtl *c) {
  if (c->inner_done) return;
  __shared__ float buf[2][kCoarseMax];
  const int I = threadIdx.x;
  const bool own = I < L.N;
  int X = 0, Y = 0, Z = 0;
  float d = 0.f, ri = 0.f, a[27];
  int nb[27];
  if (own) {
    X = I % L.nx;
    Y = (I / L.nx) % L.ny;
    Z = I / (L.nx * L.ny);
    d = A[13LL * L.N + I];
    ri = r[I];
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      a[q] = A[(long long)q * L.N + I];
      const int jx = wrap(X + q % 3 - 1, L.nx), jy = wrap(Y + (q / 3) % 3 - 1, L.ny), jz = wrap(Z + q / 9 - 1, L.nz);
      nb[q] = jx + L.nx * (jy + L.ny * jz);
    }
    buf[0][I] = d != 0.f ? kOmega * ri / d : 0.f;
  }
  __syncthreads();
  int cur = 0;
  for (int s = 1; s < kCoarseSweeps; ++s) {
    if (own) {
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 27; ++q) acc += a[q] * buf[cur][nb[q]];
      buf[cur ^ 1][I] = d != 0.f ? buf[cur][I] + kOmega * (ri - acc) / d : 0.f;
    }
    __syncthreads();
    cur ^= 1;
  }
  if (own) e[I] = buf[cur][I];
}

dim3 lgrid(const LevelDev &L, dim3 &block) {
  const Geo g{L.nx, L.ny, L.nz, L.px, L.py, L.pz, L.N};
  const Launch la = make_launch(g);
  block = la.block;
  return la.grid;
}

LevelDev level_dev(const Geo &g, const MGLevel &L) {
  return LevelDev{L.nx, L.ny, L.nz, g.px, g.py, g.pz, L.sx, L.sy, L.sz, (int)L.N};
}

}  // namespace

// build the hierarchy for the current geometry (after the link mask)
cudaError_t mg_setup(lbe_handle *h) {
  MGWork &mg = h->mg;
  mg_free(h);
  const Geo &g = h->geo;
  int nx = g.nx, ny = g.ny, nz = g.nz;
  for (int l = 1; l < kMaxLevels; ++l) {
    const bool cx = nx > 1 && (nx % 2 == 0 || !g.px), cy = ny > 1 && (ny % 2 == 0 || !g.py),
               cz = nz > 1 && (nz % 2 == 0 || !g.pz);
    if (!cx && !cy && !cz) break;
    if ((long long)nx * ny * nz <= kCoarseTarget && l > 1) break;
    nx = cx ? (nx + 1) / 2 : nx;
    ny = cy ? (ny + 1) / 2 : ny;
    nz = cz ? (nz + 1) / 2 : nz;
    MGLevel &L = mg.lv[l];
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    L.sx = cx;
    L.sy = cy;
    L.sz = cz;
    L.N = (long long)nx * ny * nz;
    mg.nlev = l + 1;
  }
  // the coarsest level must fit the one-block solve
  if (mg.nlev < 2 || mg.lv[mg.nlev - 1].N > kCoarseMax) {
    mg.nlev = 0;
    return cudaSuccess;  // plain Jacobi preconditioning
  }
  cudaError_t e = cudaMalloc(&mg.inv0, sizeof(float) * g.N);
  if (e == cudaSuccess) e = cudaMalloc(&mg.t0, sizeof(float) * g.N);
  for (int l = 1; l < mg.nlev && e == cudaSuccess; ++l) {
    MGLevel &L = mg.lv[l];
    e = cudaMalloc(&L.A, sizeof(float) * 27 * L.N);
    if (e == cudaSuccess) e = cudaMalloc(&L.r, sizeof(float) * L.N);
    if (e == cudaSuccess) e = cudaMalloc(&L.e, sizeof(float) * L.N);
  }
  if (e != cudaSuccess) {
    mg_free(h);
    return e;
  }
  const Launch L0 = make_launch(g);
  k_invdiag0<<<L0.grid, L0.block, 0, h->stream>>>(g, h->phys.selfmask, h->mask, mg.inv0);
  for (int l = 1; l < mg.nlev; ++l) {
    const LevelDev C = level_dev(g, mg.lv[l]);
    dim3 blk;
    const dim3 grd = lgrid(C, blk);
    if (l == 1)
      k_galerkin0<<<grd, blk, 0, h->stream>>>(g, h->phys.selfmask, h->mask, C, mg.lv[1].A);
    else
      k_galerkin<<<grd, blk, 0, h->stream>>>(level_dev(g, mg.lv[l - 1]), mg.lv[l - 1].A, C, mg.lv[l].A);
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
  }
  cudaFree(mg.t0);
  cudaFree(mg.inv0);
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
    void *args[9];
  };
  std::vector<Node> nodes;
  std::vector<LevelDev> lv(kMaxLevels);
  std::vector<const void *> ptr;
  ptr.reserve(512);  // no reallocation: the kernel arguments point into it
  auto P = [&](const void *v) -> void * {
    ptr.push_back(v);
    return &ptr.back();
  };
  for (int l = 1; l < nl; ++l) lv[l] = level_dev(g, mg.lv[l]);
  const void *pg = &g, *psm = &sm;
  auto cgrid = [](const LevelDev &C) { return dim3((unsigned)((C.N * 8 + 255) / 256)); };
  // down: restrictions (pre-smoothing on the fly)
  nodes.push_back(Node{(void *)k_restrict0, cgrid(lv[1]), dim3(256),
                       {(void *)pg, (void *)psm, P(h->mask), P(r0), P(mg.inv0), &lv[1], P(mg.lv[1].r), P(c)}});
  for (int l = 1; l < nl - 1; ++l)
    nodes.push_back(Node{(void *)k_restrict, cgrid(lv[l + 1]), dim3(256),
                         {&lv[l], P(mg.lv[l].A), P(mg.lv[l].r), &lv[l + 1], P(mg.lv[l + 1].r), P(c)}});
  // coarsest
  nodes.push_back(Node{(void *)k_coarsest, dim3(1), dim3(kCoarseMax),
                       {&lv[nl - 1], P(mg.lv[nl - 1].A), P(mg.lv[nl - 1].r), P(mg.lv[nl - 1].e), P(c)}});
  // up: fused prolongation + post-smoothing on the coarse levels
  for (int l = nl - 2; l >= 1; --l) {
    dim3 blk;
    const dim3 grd = lgrid(lv[l], blk);
    nodes.push_back(Node{(void *)k_post, grd, blk,
                         {&lv[l], P(mg.lv[l].A), P(mg.lv[l].r), &lv[l + 1], P(mg.lv[l + 1].e), P(mg.lv[l].e),
                          P(c)}});
  }
  // finest level
  nodes.push_back(Node{(void *)k_prolong0, L0.grid, L0.block,
                       {(void *)pg, P(h->mask), P(r0), P(mg.inv0), &lv[1], P(mg.lv[1].e), P(mg.t0), P(c)}});
  nodes.push_back(Node{(void *)k_post0, L0.grid, L0.block,
                       {(void *)pg, (void *)psm, P(h->mask), P(r0), P(mg.inv0), P(mg.t0), P(u0), P(c)}});
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
