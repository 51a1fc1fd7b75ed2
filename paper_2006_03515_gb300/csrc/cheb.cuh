// Chebyshev-node representation (the black-box FMM of Fong and Darve, 2009), used in
// place of the paper's equivalent and check surfaces when the plan asks for it.
//
// Per axis the p nodes are xbar_n = cos((2n + 1) pi / (2p)), n = 0..p-1, on [-1, 1]; a box
// of centre c and half-width r carries values at c + r (xbar_nx, xbar_ny, xbar_nz), node
// index m = nx + p ny + p^2 nz. The interpolation weight of node n at x is
//   S(x, xbar_n) = 1/p + (2/p) sum_{k=1}^{p-1} T_k(x) T_k(xbar_n),
// the 3-D weight the product over the axes. The plan stores tab[n][k] = c_k T_k(xbar_n)
// (c_0 = 1/p, c_k = 2/p), row stride kChebTab, so that S(x, xbar_n) = sum_k tab[n][k] T_k(x).
#pragma once

namespace kifmm {

constexpr int kChebMaxP = 10;   // largest p the plan accepts
constexpr int kChebTab = 10;    // row stride of the weight table

// T_0(x) .. T_{p-1}(x) by the three-term recurrence (entries >= p are left unset).
template <class F>
__device__ __forceinline__ void cheb_T(F x, int p, F (&t)[kChebMaxP]) {
    t[0] = F(1);
    t[1] = x;
#pragma unroll
    for (int k = 2; k < kChebMaxP; ++k)
        if (k < p) t[k] = F(2) * x * t[k - 1] - t[k - 2];
}

// S(x, xbar_n) from T_k(x) and the weight table row of node n.
template <class F>
__device__ __forceinline__ F cheb_S(const F (&t)[kChebMaxP], int p, const F* row) {
    F s = row[0];
#pragma unroll
    for (int k = 1; k < kChebMaxP; ++k)
        if (k < p) s += row[k] * t[k];
    return s;
}

}  // namespace kifmm
