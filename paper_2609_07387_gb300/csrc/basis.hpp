// Monomial basis of the reconstruction polynomial (Eq. 3): psi_k = xi^e_k,
// xi = (x - x_i)/h_i, h_i = |V_i|^(1/3), k = 0 .. K(r) - 1 with
// K(r) = (r+1)(r+2)(r+3)/6 - 1 non-constant modes (3, 9, 19, 34 for r = 1..4).
// Shared by the host precompute and the kernels.
#pragma once

#ifdef __CUDACC__
#define UCNS_HD __host__ __device__
#else
#define UCNS_HD
#endif

namespace ucns {

constexpr int kMaxOrder = 4;

UCNS_HD constexpr int basis_count(int r) { return (r + 1) * (r + 2) * (r + 3) / 6 - 1; }

// exponent of coordinate d in basis monomial k: the nine of P2 in the order
// x y z xx yy zz xy xz yz, then the cubics and the quartics, each by
// descending power of x, then of y
UCNS_HD constexpr int basis_exp(int k, int d) {
  constexpr signed char t[34][3] = {
      {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1},
      {3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1}, {1, 0, 2}, {0, 3, 0}, {0, 2, 1}, {0, 1, 2}, {0, 0, 3},
      {4, 0, 0}, {3, 1, 0}, {3, 0, 1}, {2, 2, 0}, {2, 1, 1}, {2, 0, 2}, {1, 3, 0}, {1, 2, 1}, {1, 1, 2}, {1, 0, 3},
      {0, 4, 0}, {0, 3, 1}, {0, 2, 2}, {0, 1, 3}, {0, 0, 4}};
  return t[k][d];
}

UCNS_HD constexpr int basis_degree(int k) { return basis_exp(k, 0) + basis_exp(k, 1) + basis_exp(k, 2); }

}  // namespace ucns
