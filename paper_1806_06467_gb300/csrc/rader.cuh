// rader.cuh -- the shape of the Rader stage for a prime radix (shared by the table builder and
// the packed-pair mixed-radix engine).
//
// Rader's algorithm turns an R-point DFT, R prime, into a cyclic convolution of length
// L = R - 1: with g a primitive root mod R, X[g^-p] = x[0] + sum_q x[g^q] W_R^(g^(q-p)). The
// convolution runs as two length-L DFTs with L = L1 x L2, L1 a power of two up to 16 and L2 odd
// up to 15 (41: L = 40 = 8 x 5), so both factors are butterflies the engine has.
#pragma once

namespace coro {

// Smallest primitive root of the prime r (0 when r is not prime or below 3).
__host__ __device__ constexpr int rader_root(int r) {
    if (r < 3) return 0;
    for (int d = 2; d * d <= r; ++d)
        if (r % d == 0) return 0;
    for (int g = 2; g < r; ++g) {
        int x = 1, k = 0;
        do {
            x = x * g % r;
            ++k;
        } while (x != 1);
        if (k == r - 1) return g;
    }
    return 0;
}

// L1 of the Rader split of the prime radix r (the power-of-two factor of r - 1, at most 16,
// with an odd cofactor L2 = (r - 1) / L1 of at most 15), or 0 when r takes no Rader stage
// (r up to 13, where the pair-sum DFT is cheaper, or no such split).
__host__ __device__ constexpr int rader_l1(int r) {
    if (r <= 13 || rader_root(r) == 0) return 0;
    int l1 = 1;
    while ((r - 1) % (2 * l1) == 0 && 2 * l1 <= 16) l1 *= 2;
    const int l2 = (r - 1) / l1;
    return (l2 % 2 == 1 && l2 <= 15) ? l1 : 0;
}

// g^e mod r for small e (the exponent is a loop count).
__host__ __device__ constexpr int rader_pow(int g, int e, int r) {
    int x = 1;
    for (int i = 0; i < e; ++i) x = x * g % r;
    return x;
}

// Entries of the Rader tables appended after the twiddle blocks for a last radix r: w_L^m
// (m < L), then B_f[k] and B_i[k] (k < L), the length-L DFTs of b_m = W_r^(+-g^-m) divided by L
// (forward and inverse transform direction).
__host__ __device__ constexpr int rader_table_len(int r) { return rader_l1(r) ? 3 * (r - 1) : 0; }

}  // namespace coro
