// Host check of the multigrid's coarsest-level inverse (mgd::coarse_inverse
// in mg.cu): no GPU is used.  Prints one line per case; the Python test
// parses it.
//   spd:      a 4x4x6 level (x, y periodic, z bounded) with a shifted 7-point
//             operator and one node with zero diagonal; A inv = I on the
//             active nodes, zero row and column for the inactive one
//   singular: the periodic 6-neighbour Laplacian on 4x4x4 (constant null
//             space): rejected
#include <cstdio>
#include <vector>

#include "../../paper_1907_04732_gb300/csrc/mg.cu"

using lbe::mgd::d27;
using lbe::mgd::MgLevel;

static int wrapi(int c, int n) { return (c % n + n) % n; }

int main() {
  const int nx = 4, ny = 4, nz = 6, N = nx * ny * nz, dead = 50;
  MgLevel L{nx, ny, nz, 1, 1, 1, N, N};
  std::vector<float> A(27 * (size_t)N, 0.f);
  const int faces[6] = {d27(-1, 0, 0), d27(1, 0, 0), d27(0, -1, 0), d27(0, 1, 0), d27(0, 0, -1), d27(0, 0, 1)};
  const int fz[6] = {0, 0, 0, 0, -1, 1};
  for (int I = 0; I < N; ++I) {
    const int Z = I / (nx * ny);
    if (I == dead) continue;
    A[13 * N + I] = 6.5f;
    for (int f = 0; f < 6; ++f) {
      const int z2 = Z + fz[f];
      if (z2 < 0 || z2 >= nz) continue;
      const int X = I % nx, Y = (I / nx) % ny;
      const int q = faces[f];
      const int J = wrapi(X + q % 3 - 1, nx) + nx * (wrapi(Y + (q / 3) % 3 - 1, ny) + ny * z2);
      if (J != dead) A[q * N + I] = -1.f;
    }
  }
  std::vector<float> inv;
  const bool ok = lbe::mgd::coarse_inverse(L, A, inv);
  double err = 0.0;
  bool dead_zero = true;
  for (int c = 0; c < N; ++c) {
    dead_zero = dead_zero && inv[(size_t)dead * N + c] == 0.f && inv[(size_t)c * N + dead] == 0.f;
    if (c == dead) continue;
    for (int I = 0; I < N; ++I) {
      if (I == dead) continue;
      const int X = I % nx, Y = (I / nx) % ny, Z = I / (nx * ny);
      double s = 0.0;
      for (int q = 0; q < 27; ++q) {
        const float a = A[q * N + I];
        if (a == 0.f) continue;
        const int J = wrapi(X + q % 3 - 1, nx) + nx * (wrapi(Y + (q / 3) % 3 - 1, ny) + ny * (Z + q / 9 - 1));
        s += a * (double)inv[(size_t)J * N + c];
      }
      const double want = I == c ? 1.0 : 0.0;
      err = std::max(err, std::fabs(s - want));
    }
  }
  std::printf("spd ok=%d err=%.3e dead_zero=%d\n", ok ? 1 : 0, err, dead_zero ? 1 : 0);

  const int m = 4, M = m * m * m;
  MgLevel P{m, m, m, 1, 1, 1, M, M};
  std::vector<float> B(27 * (size_t)M, 0.f);
  for (int I = 0; I < M; ++I) {
    B[13 * M + I] = 6.f;
    for (int f = 0; f < 6; ++f) B[faces[f] * M + I] = -1.f;
  }
  std::printf("singular ok=%d\n", lbe::mgd::coarse_inverse(P, B, inv) ? 1 : 0);
  return 0;
}
