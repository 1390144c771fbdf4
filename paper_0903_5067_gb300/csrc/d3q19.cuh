// D3Q19 lattice and moment basis for the CUDA path.
//
// Velocities (Sec. II B of Pham, Schiller, Prakash, Duenweg): the rest particle, the 6
// nearest and the 12 next-nearest neighbours of the simple cubic lattice, with weights 1/3,
// 1/18, 1/36 and c_s^2 = 1/3 in lattice units.  The order below is the library's ABI order;
// velocities 2p+1 and 2p+2 (p = 0..8) are opposite.
//
// Moment basis: the orthogonal D3Q19 basis of Duenweg, Schiller & Ladd (2007), which the
// paper cites for its fully thermalized model.  Every table is produced at compile time
// from the basis polynomials evaluated on the velocities, so the kernels' fully unrolled
// transforms reduce to additions with small integer coefficients.
#pragma once

namespace gblb {

constexpr int Q = 19;
constexpr int NPAIR = 9;

__host__ __device__ constexpr int cx(int i) {
  constexpr int v[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
  return v[i];
}
__host__ __device__ constexpr int cy(int i) {
  constexpr int v[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
  return v[i];
}
__host__ __device__ constexpr int cz(int i) {
  constexpr int v[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
  return v[i];
}
__host__ __device__ constexpr int c2(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }

// the components of all 19 velocities packed two bits each (c + 1), for loops over i that
// are not unrolled: component = ((packed >> 2i) & 3) - 1
__host__ __device__ constexpr unsigned long long pack_component(int comp) {
  unsigned long long p = 0;
  for (int i = 0; i < Q; ++i) {
    const int c = comp == 0 ? cx(i) : (comp == 1 ? cy(i) : cz(i));
    p |= (unsigned long long)(c + 1) << (2 * i);
  }
  return p;
}
__host__ __device__ constexpr int unpack_component(unsigned long long packed, int i) {
  return (int)((packed >> (2 * i)) & 3ull) - 1;
}

// weight numerator over 36: 12, 2, 1
__host__ __device__ constexpr int w36(int i) { return c2(i) == 0 ? 12 : (c2(i) == 1 ? 2 : 1); }

// e_k(c_i): value of basis polynomial k on velocity i
__host__ __device__ constexpr int basis(int k, int i) {
  const int x = cx(i), y = cy(i), z = cz(i), s = c2(i);
  switch (k) {
    case 0: return 1;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return s - 1;
    case 5: return 3 * x * x - s;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return y * z;
    case 9: return x * z;
    case 10: return (3 * s - 5) * x;
    case 11: return (3 * s - 5) * y;
    case 12: return (3 * s - 5) * z;
    case 13: return (y * y - z * z) * x;
    case 14: return (z * z - x * x) * y;
    case 15: return (x * x - y * y) * z;
    case 16: return 3 * s * s - 6 * s + 1;
    case 17: return (2 * s - 3) * (3 * x * x - s);
    case 18: return (2 * s - 3) * (y * y - z * z);
  }
  return 0;
}

// odd polynomials change sign under c -> -c
__host__ __device__ constexpr bool odd_mode(int k) {
  return (k >= 1 && k <= 3) || (k >= 10 && k <= 15);
}

// b_k = sum_i w_i e_k(c_i)^2, as a rational num/den (den 36 * 1)
__host__ __device__ constexpr int norm36(int k) {
  int acc = 0;
  for (int i = 0; i < Q; ++i) acc += w36(i) * basis(k, i) * basis(k, i);
  return acc;  // b_k = acc / 36
}

}  // namespace gblb
