// Per-node arithmetic of the geometric multigrid preconditioner of the FP32
// Poisson correction solve, shared by the single-lattice V-cycle (mg.cu) and
// the batched one (batch.cu).
//
//   hierarchy   level 0 is the lattice with the modified-Laplacian operator
//               of Eq. DiscreteLaplacianModif on fluid nodes; level l+1
//               aggregates 2x2x2 nodes of level l (an axis of one node is
//               kept) and carries the Galerkin operator A_{l+1} = P^T A_l P
//               of the piecewise-constant prolongation P: 27 points, exact
//               for any electrode shape, solid nodes being Dirichlet zeros
//               of the correction
//   smoother    weighted Jacobi, one sweep before and one after the coarse
//               correction (the same on both sides, so the preconditioner
//               is symmetric)
//   correction  e += alpha P e_c, alpha > 1 compensating the stiffness of
//               piecewise-constant coarse spaces
//   coarsest    solved exactly with its inverse (formed on the host at
//               set-up, coarse_inverse) where the operator is positive
//               definite, else a fixed number of Jacobi sweeps in one
//               thread block
//
// A coarse level is an MgLevel; its operator is stored component-major with
// component stride S (S = N for one lattice, the level's total node count
// when several lattices are concatenated), and every pointer handed to these
// functions is already offset to the lattice's first node of that level.
#pragma once

#include <vector>

#include "lbe_internal.cuh"

namespace lbe {
namespace mgd {

// Smoother and correction constants (compile-time).  Measured on the
// electro-osmosis, porous-electrode and coaxial lattices (CG iterations per
// step, omega / alpha): 0.7/1.6 10.7, 14.9, 12.2; 0.9/1.8 7.6, 14.0, 9.5;
// 1.0/1.8 7.0, 12.2, 8.0; 1.1/1.8 6.0, 10.3, 7.9; at 1.15/1.8 the V-cycle
// stops being positive definite on the porous lattice (the CG stalls).
// The Jacobi-scaled 19-point operator has its largest eigenvalue near 4/3
// (smoothing needs omega below ~1.5), and alpha = 2 is where the coarse
// correction stops contracting: 1.0/1.8 keeps a margin from both.
#ifndef LBE_MG_OMEGA
#define LBE_MG_OMEGA 1.0f
#endif
#ifndef LBE_MG_ALPHA
#define LBE_MG_ALPHA 1.8f
#endif
#ifndef LBE_MG_COARSE_SWEEPS
#define LBE_MG_COARSE_SWEEPS 32
#endif
constexpr float kOmega = LBE_MG_OMEGA;               // Jacobi weight
constexpr float kAlpha = LBE_MG_ALPHA;               // coarse-correction scaling
constexpr int kCoarseSweeps = LBE_MG_COARSE_SWEEPS;  // Jacobi sweeps on the coarsest level
constexpr int kCoarseTarget = 256; // coarsening stops at or below this size
constexpr int kCoarseMax = 1024;   // the coarsest solve owns one node per thread

struct MgLevel {
  int nx, ny, nz;
  int sx, sy, sz;  // 1 when this level halves the axis of the finer level
  int N;
  long long S;     // component stride of the operator array
};

// Shapes of the coarse levels of an nx x ny x nz lattice: every axis longer
// than one node is halved (rounding up; the last aggregate of an odd axis
// holds one node, on a periodic axis it neighbours the first one) until the
// level has at most kCoarseTarget nodes.  Returns the level count (including
// level 0), or 0 when the coarsest level would not fit the one-block solve.
inline int level_shapes(int nx, int ny, int nz, MgLevel out[kMaxLevels]) {
  int nlev = 1;
  for (int l = 1; l < kMaxLevels; ++l) {
    const bool cx = nx > 1, cy = ny > 1, cz = nz > 1;
    if (!cx && !cy && !cz) break;
    if ((long long)nx * ny * nz <= kCoarseTarget && l > 1) break;
    nx = cx ? (nx + 1) / 2 : nx;
    ny = cy ? (ny + 1) / 2 : ny;
    nz = cz ? (nz + 1) / 2 : nz;
    out[l] = MgLevel{nx, ny, nz, cx, cy, cz, nx * ny * nz, (long long)nx * ny * nz};
    nlev = l + 1;
  }
  if (nlev < 2 || out[nlev - 1].N > kCoarseMax) return 0;
  return nlev;
}

__host__ __device__ constexpr int d27(int dx, int dy, int dz) { return (dx + 1) + 3 * ((dy + 1) + 3 * (dz + 1)); }

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

__device__ __forceinline__ int agg_index(const MgLevel &C, int x, int y, int z) {
  return (x >> C.sx) + C.nx * ((y >> C.sy) + C.ny * (z >> C.sz));
}

__device__ __forceinline__ void level_coords(const MgLevel &L, int I, int &X, int &Y, int &Z) {
  X = I % L.nx;
  Y = (I / L.nx) % L.ny;
  Z = I / (L.nx * L.ny);
}

// child ch (0..7) of coarse node (X,Y,Z) in the finer level of size n*;
// false when the child does not exist
__device__ __forceinline__ bool child_of(const MgLevel &C, int X, int Y, int Z, int ch, int fnx, int fny, int fnz,
                                         int &x, int &y, int &z) {
  const int ax = ch & 1, ay = (ch >> 1) & 1, az = ch >> 2;
  if ((ax && !C.sx) || (ay && !C.sy) || (az && !C.sz)) return false;
  x = (X << C.sx) + ax;
  y = (Y << C.sy) + ay;
  z = (Z << C.sz) + az;
  return x < fnx && y < fny && z < fnz;
}

// --- set-up ------------------------------------------------------------------
// Galerkin row of coarse node (X,Y,Z) of level 1 from the fine lattice
// (mask-defined operator); mask points at the lattice's node 0
__device__ __forceinline__ void galerkin0_row(const Geo &g, uint32_t selfmask, const uint32_t *__restrict__ mask,
                                              const MgLevel &C, int X, int Y, int Z, float a[27]) {
#pragma unroll
  for (int d = 0; d < 27; ++d) a[d] = 0.f;
  for (int c = 0; c < 8; ++c) {
    int x, y, z;
    if (!child_of(C, X, Y, Z, c, g.nx, g.ny, g.nz, x, y, z)) continue;
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
}

// Galerkin row of coarse node (X,Y,Z) of level l+1 from level l (27-point)
__device__ __forceinline__ void galerkin_row(const MgLevel &F, const float *__restrict__ AF, const MgLevel &C, int X,
                                             int Y, int Z, float a[27]) {
#pragma unroll
  for (int d = 0; d < 27; ++d) a[d] = 0.f;
  for (int c = 0; c < 8; ++c) {
    int x, y, z;
    if (!child_of(C, X, Y, Z, c, F.nx, F.ny, F.nz, x, y, z)) continue;
    const int i = x + F.nx * (y + F.ny * z);
    if (AF[13 * F.S + i] == 0.f) continue;  // inactive node
    for (int d = 0; d < 27; ++d) {
      const float v = AF[d * F.S + i];
      if (v == 0.f) continue;
      const int jx = wrap(x + d % 3 - 1, F.nx), jy = wrap(y + (d / 3) % 3 - 1, F.ny), jz = wrap(z + d / 9 - 1, F.nz);
      const int dx = rel(jx >> C.sx, X, C.nx), dy = rel(jy >> C.sy, Y, C.ny), dz = rel(jz >> C.sz, Z, C.nz);
      a[d27(dx, dy, dz)] += v;
    }
  }
}

// --- V-cycle -----------------------------------------------------------------
__device__ __forceinline__ float sum8(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  return v;
}

// coarsest level: kCoarseSweeps weighted Jacobi sweeps from zero by one
// block of kCoarseMax threads, one node per thread, iterates in buf
__device__ __forceinline__ void coarsest_solve(const MgLevel &L, const float *__restrict__ A,
                                               const float *__restrict__ r, float *__restrict__ e,
                                               float (*buf)[kCoarseMax]) {
  const int I = threadIdx.x;
  const bool own = I < L.N;
  float d = 0.f, ri = 0.f, a[27];
  int nb[27];
  if (own) {
    int X, Y, Z;
    level_coords(L, I, X, Y, Z);
    d = A[13 * L.S + I];
    ri = r[I];
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      a[q] = A[q * L.S + I];
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


// a coarse node's restricted residual rc and pre-smoothed iterate
// zc = omega rc/diag
__device__ __forceinline__ void store_coarse(const MgLevel &C, int I, float v, const float *__restrict__ AC,
                                             float *__restrict__ rc, float *__restrict__ zc) {
  const float d = AC[13 * C.S + I];
  rc[I] = v;
  zc[I] = d != 0.f ? kOmega * v / d : 0.f;
}

// --- forms with integer link weights and a stored pre-smoothed iterate -------
// The modified Laplacian's link weights 1/3 (axis) and 1/6 (diagonal) are
// 2/6 and 1/6: sums of weights are integers over 6, and a node's diagonal
// 6 * diag = sum over non-self links of (2 - fluid) * (2 axis, 1 diagonal)
// follows from two population counts of its link mask.
__host__ __device__ constexpr uint32_t axis_links() {
  uint32_t m = 0;
  for (int l = 1; l < kQ; ++l)
    if (c2_of(l) == 1) m |= 1u << (l - 1);
  return m;
}
__host__ __device__ constexpr uint32_t diag_links() {
  uint32_t m = 0;
  for (int l = 1; l < kQ; ++l)
    if (c2_of(l) == 2) m |= 1u << (l - 1);
  return m;
}

// 6 * diagonal of a fluid node's row
__device__ __forceinline__ int diag6(uint32_t m, uint32_t selfmask) {
  const uint32_t ax = axis_links() & ~selfmask, dg = diag_links() & ~selfmask;
  return 2 * (2 * __popc(ax) + __popc(dg)) - (2 * __popc(m & ax) + __popc(m & dg));
}

// 6 * sum over fluid links of weight * v[neighbour]; every neighbour is
// read (a zero weight drops it) so that the loads do not wait for the mask.
// A node with all links fluid takes the same fmaf sequence without the
// per-link weight tests.
__device__ __forceinline__ float nbsum6(uint32_t m, uint32_t selfmask, const Offs &o, int i,
                                        const float *__restrict__ v) {
  const float *__restrict__ vi = v + i;
  float s = 0.f;
  if (all_links(m, selfmask)) {
#pragma unroll
    for (int l = 1; l < kQ; ++l) s = fmaf(c2_of(l) == 1 ? 2.f : 1.f, vi[o.at(cx_of(l), cy_of(l), cz_of(l))], s);
    return s;
  }
#pragma unroll
  for (int l = 1; l < kQ; ++l) {
    const uint32_t b = 1u << (l - 1);
    const float vj = vi[o.at(cx_of(l), cy_of(l), cz_of(l))];
    const float wl = ((m & b) && !(selfmask & b)) ? (c2_of(l) == 1 ? 2.f : 1.f) : 0.f;
    s = fmaf(wl, vj, s);
  }
  return s;
}

// residual of a 27-point level after pre-smoothing, the pre-smoothed iterate
// z = omega r/diag being stored: r - A z at (X,Y,Z)
__device__ __forceinline__ float presmoothed_res_z(const MgLevel &L, const float *__restrict__ A,
                                                   const float *__restrict__ r, const float *__restrict__ z, int X,
                                                   int Y, int Z) {
  const int I = X + L.nx * (Y + L.ny * Z);
  if (A[13 * L.S + I] == 0.f) return 0.f;
  float s = 0.f;
#pragma unroll
  for (int d = 0; d < 27; ++d) {  // a zero coefficient adds nothing; no branch
    const float a = A[d * L.S + I];
    const int jx = wrap(X + d % 3 - 1, L.nx), jy = wrap(Y + (d / 3) % 3 - 1, L.ny), jz = wrap(Z + d / 9 - 1, L.nz);
    s = fmaf(a, z[jx + L.nx * (jy + L.ny * jz)], s);
  }
  return r[I] - s;
}

// fused prolongation + post-smoothing with the stored iterate:
// e = z + alpha P e_c, out = e + omega (r - A e)/diag
__device__ __forceinline__ float post_value_z(const MgLevel &L, const float *__restrict__ A,
                                             const float *__restrict__ r, const float *__restrict__ z,
                                             const MgLevel &C, const float *__restrict__ ec, int X, int Y, int Z) {
  const int I = X + L.nx * (Y + L.ny * Z);
  const float d = A[13 * L.S + I];
  if (d == 0.f) return 0.f;
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 27; ++q) {  // a zero coefficient adds nothing; no branch
    const float a = A[q * L.S + I];
    const int jx = wrap(X + q % 3 - 1, L.nx), jy = wrap(Y + (q / 3) % 3 - 1, L.ny), jz = wrap(Z + q / 9 - 1, L.nz);
    const float ej = fmaf(kAlpha, ec[agg_index(C, jx, jy, jz)], z[jx + L.nx * (jy + L.ny * jz)]);
    s = fmaf(a, ej, s);
  }
  const float e = fmaf(kAlpha, ec[agg_index(C, X, Y, Z)], z[I]);
  return e + kOmega * (r[I] - s) / d;
}

// host (mg.cu): inverse of a coarsest level's operator, A27 its 27-point
// rows [27][L.N]; inv [L.N][L.N] with zero rows and columns for the nodes
// with a zero diagonal; false when the operator is not symmetric positive
// definite to working accuracy
bool coarse_inverse(const MgLevel &L, const std::vector<float> &A27, std::vector<float> &inv);

}  // namespace mgd
}  // namespace lbe
