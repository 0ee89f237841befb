// Compile-time register FFTs shared by the plane-stage kernels (xz_reg.cu: float,
// xz_reg64.cu: double).
//
// The FFT is a decimation-in-frequency Cooley-Tukey recursion with radices
// 4, 3 and 2 fully unrolled at compile time: inputs in natural order, outputs
// in digit-reversed positions resolved by a compile-time index map, twiddles
// as compile-time constants (sine and cosine evaluated by Taylor series at
// compile time). Trivial twiddles (w^0) cost nothing; outputs a caller never
// reads are removed by the compiler as dead code.
#pragma once

#include <utility>

#include "sp_internal.h"

namespace fftreg {

// ------------------------------------------------- compile-time trigonometry
constexpr double kPi = 3.14159265358979323846264338327950288;

// Taylor series about 0; |x| <= pi/4 after the reduction below (30 terms is
// far below double rounding there)
__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
// cos and sin of 2 pi k / n for integers, reduced exactly by octant symmetry
__host__ __device__ constexpr double cos2pi(long k, long n) {
  long m = ((k % n) + n) % n;            // angle 2 pi m / n in [0, 2 pi)
  if (8 * m <= n) return taylor_cos(2.0 * kPi * (double)m / (double)n);
  if (8 * m <= 3 * n) return taylor_sin(2.0 * kPi * (double)(n - 4 * m) / (4.0 * n));   // cos(pi/2 - t)
  if (8 * m <= 5 * n) return -taylor_cos(2.0 * kPi * (double)(2 * m - n) / (2.0 * n));  // -cos(t - pi)
  if (8 * m <= 7 * n) return -taylor_sin(2.0 * kPi * (double)(3 * n - 4 * m) / (4.0 * n));
  return taylor_cos(2.0 * kPi * (double)(n - m) / (double)n);
}
__host__ __device__ constexpr double sin2pi(long k, long n) { return cos2pi(n - 4 * k, 4 * n); }  // sin t = cos(pi/2 - t)

// -------------------------------------------------------------- radix plans
template <int N> struct Plan;
template <> struct Plan<2> { using type = std::integer_sequence<int, 2>; };
template <> struct Plan<3> { using type = std::integer_sequence<int, 3>; };
template <> struct Plan<4> { using type = std::integer_sequence<int, 4>; };
template <> struct Plan<8> { using type = std::integer_sequence<int, 4, 2>; };
template <> struct Plan<12> { using type = std::integer_sequence<int, 4, 3>; };
template <> struct Plan<16> { using type = std::integer_sequence<int, 4, 4>; };
template <> struct Plan<24> { using type = std::integer_sequence<int, 4, 3, 2>; };
template <> struct Plan<32> { using type = std::integer_sequence<int, 4, 4, 2>; };
template <> struct Plan<48> { using type = std::integer_sequence<int, 4, 4, 3>; };
template <> struct Plan<64> { using type = std::integer_sequence<int, 4, 4, 4>; };

// position of output frequency f after the DIF recursion with radices P0, Pr...
template <int N, int P0, int... Pr>
__host__ __device__ constexpr int dif_pos(int f) {
  constexpr int M = N / P0;
  if constexpr (sizeof...(Pr) == 0) {
    return (f % P0) * M;
  } else {
    return (f % P0) * M + dif_pos<M, Pr...>(f / P0);
  }
}
template <int N, int... P>
__host__ __device__ constexpr int out_pos_impl(int f, std::integer_sequence<int, P...>) { return dif_pos<N, P...>(f); }
template <int N>
__host__ __device__ constexpr int out_pos(int f) { return out_pos_impl<N>(f, typename Plan<N>::type{}); }

// y_d = sum_r x_r w_P^{r d}, w_P = exp(SGN 2 pi i / P)
template <int P, int SGN, typename T>
__device__ __forceinline__ void bfly(C2<T>* v) {
  if constexpr (P == 2) {
    const C2<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  } else if constexpr (P == 3) {
    constexpr T h3 = (T)(0.86602540378443864676 * SGN);
    const C2<T> t1 = v[1] + v[2];
    const C2<T> t2 = mul_is(v[1] - v[2], h3);
    const C2<T> m = v[0] - scl(t1, (T)0.5);
    v[0] = v[0] + t1;
    v[1] = m + t2;
    v[2] = m - t2;
  } else {
    const C2<T> a = v[0] + v[2], b = v[0] - v[2];
    const C2<T> c = v[1] + v[3], d = mul_is(v[1] - v[3], (T)SGN);
    v[0] = a + c;
    v[2] = a - c;
    v[1] = b + d;
    v[3] = b - d;
  }
}

template <typename T, int NT, int N, int OFF, int SGN, int P0, int... Pr>
__device__ __forceinline__ void dif(C2<T> (&x)[NT]);

template <typename T, int NT, int M, int OFF, int SGN, int... Pr, int... D>
__device__ __forceinline__ void dif_blocks(C2<T> (&x)[NT], std::integer_sequence<int, D...>) {
  (dif<T, NT, M, OFF + D * M, SGN, Pr...>(x), ...);
}

// multiply by w_N^{SGN k} (a compile-time constant; k = 0 is the identity). Quarter turns
// (w = -1, +-i) are sign changes and swaps: written as products with 0 and 1 they would
// still cost two FMAs, since x * 0 cannot be dropped under IEEE rules.
template <typename T, int N, int SGN, long K>
__device__ __forceinline__ C2<T> twiddle(C2<T> y) {
  constexpr long Kr = ((K % N) + N) % N;
  if constexpr (Kr == 0) {
    return y;
  } else if constexpr (4 * Kr == 2 * N) {  // w = -1
    return mk(-y.x, -y.y);
  } else if constexpr (4 * Kr == N || 4 * Kr == 3 * N) {  // w = i s, s = +-1
    constexpr int s = (4 * Kr == N ? 1 : -1) * SGN;
    if constexpr (s > 0) return mk(-y.y, y.x);
    else return mk(y.y, -y.x);
  } else {
    constexpr T wc = (T)cos2pi(K, N);
    constexpr T ws = (T)(SGN * sin2pi(K, N));
    return mk(y.x * wc - y.y * ws, y.x * ws + y.y * wc);
  }
}

// twiddle by w_N^{m d} (a compile-time constant) and store at position OFF + m + d M
template <typename T, int NT, int N, int OFF, int SGN, int M, int m, int d>
__device__ __forceinline__ void tw_store(C2<T> (&x)[NT], C2<T> y) {
  x[OFF + m + d * M] = twiddle<T, N, SGN, (long)m * d>(y);
}

template <typename T, int NT, int N, int OFF, int SGN, int P0, int M, int m, int... D>
__device__ __forceinline__ void dif_col(C2<T> (&x)[NT], std::integer_sequence<int, D...>) {
  C2<T> v[P0] = {x[OFF + m + D * M]...};
  bfly<P0, SGN>(v);
  (tw_store<T, NT, N, OFF, SGN, M, m, D>(x, v[D]), ...);
}

template <typename T, int NT, int N, int OFF, int SGN, int P0, int M, int... Ms>
__device__ __forceinline__ void dif_cols(C2<T> (&x)[NT], std::integer_sequence<int, Ms...>) {
  (dif_col<T, NT, N, OFF, SGN, P0, M, Ms>(x, std::make_integer_sequence<int, P0>{}), ...);
}

// one decimation-in-frequency level on positions [OFF, OFF + N), then recurse
// on the P0 blocks of length M = N / P0
template <typename T, int NT, int N, int OFF, int SGN, int P0, int... Pr>
__device__ __forceinline__ void dif(C2<T> (&x)[NT]) {
  constexpr int M = N / P0;
  dif_cols<T, NT, N, OFF, SGN, P0, M>(x, std::make_integer_sequence<int, M>{});
  if constexpr (sizeof...(Pr) > 0) dif_blocks<T, NT, M, OFF, SGN, Pr...>(x, std::make_integer_sequence<int, P0>{});
}

template <typename T, int N, int SGN, int... P>
__device__ __forceinline__ void fft_impl(C2<T> (&x)[N], std::integer_sequence<int, P...>) {
  dif<T, N, N, 0, SGN, P...>(x);
}
// in-register FFT: natural-order input, output frequency f at x[out_pos<N>(f)]
template <int N, int SGN, typename T>
__device__ __forceinline__ void fft_reg(C2<T> (&x)[N]) {
  fft_impl<T, N, SGN>(x, typename Plan<N>::type{});
}

}  // namespace fftreg
