// Small device helpers shared by the kernel translation units.
#pragma once

#include <cuda_runtime.h>

// sum_c w[c * ws] x[c * xs] with four independent partial sums (real w, complex x):
// eight independent FMA chains per thread hide the FP64 latency
__device__ __forceinline__ double2 dot4(const double* __restrict__ w, int ws, const double2* x, int xs, int n) {
  double2 s0 = make_double2(0.0, 0.0), s1 = s0, s2 = s0, s3 = s0;
  int c = 0;
  for (; c + 4 <= n; c += 4) {
    const double w0 = __ldg(w + (size_t)c * ws), w1 = __ldg(w + (size_t)(c + 1) * ws),
                 w2 = __ldg(w + (size_t)(c + 2) * ws), w3 = __ldg(w + (size_t)(c + 3) * ws);
    const double2 x0 = x[c * xs], x1 = x[(c + 1) * xs], x2 = x[(c + 2) * xs], x3 = x[(c + 3) * xs];
    s0.x = fma(w0, x0.x, s0.x);
    s0.y = fma(w0, x0.y, s0.y);
    s1.x = fma(w1, x1.x, s1.x);
    s1.y = fma(w1, x1.y, s1.y);
    s2.x = fma(w2, x2.x, s2.x);
    s2.y = fma(w2, x2.y, s2.y);
    s3.x = fma(w3, x3.x, s3.x);
    s3.y = fma(w3, x3.y, s3.y);
  }
  for (; c < n; ++c) {
    const double w0 = __ldg(w + (size_t)c * ws);
    const double2 x0 = x[c * xs];
    s0.x = fma(w0, x0.x, s0.x);
    s0.y = fma(w0, x0.y, s0.y);
  }
  return make_double2((s0.x + s1.x) + (s2.x + s3.x), (s0.y + s1.y) + (s2.y + s3.y));
}


// sum_c w[c * ws] x[c] with complex w and x: the real and imaginary parts of each
// product go to separate partial sums, eight independent FMA chains per thread
__device__ __forceinline__ double2 cdot4(const double2* __restrict__ w, int ws, const double2* x, int n) {
  double2 s0 = make_double2(0.0, 0.0), s1 = s0, s2 = s0, s3 = s0;
  int c = 0;
  for (; c + 2 <= n; c += 2) {
    const double2 w0 = __ldg(w + (size_t)c * ws), w1 = __ldg(w + (size_t)(c + 1) * ws);
    const double2 x0 = x[c], x1 = x[c + 1];
    s0.x = fma(w0.x, x0.x, s0.x);
    s1.x = fma(-w0.y, x0.y, s1.x);
    s0.y = fma(w0.x, x0.y, s0.y);
    s1.y = fma(w0.y, x0.x, s1.y);
    s2.x = fma(w1.x, x1.x, s2.x);
    s3.x = fma(-w1.y, x1.y, s3.x);
    s2.y = fma(w1.x, x1.y, s2.y);
    s3.y = fma(w1.y, x1.x, s3.y);
  }
  if (c < n) {
    const double2 w0 = __ldg(w + (size_t)c * ws);
    const double2 x0 = x[c];
    s0.x = fma(w0.x, x0.x, s0.x);
    s1.x = fma(-w0.y, x0.y, s1.x);
    s0.y = fma(w0.x, x0.y, s0.y);
    s1.y = fma(w0.y, x0.x, s1.y);
  }
  return make_double2((s0.x + s1.x) + (s2.x + s3.x), (s0.y + s1.y) + (s2.y + s3.y));
}
