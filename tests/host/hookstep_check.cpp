// Drives the host trust-region solver of the Newton-GMRES-hookstep (hookstep.h) for the CPU
// tests: reads k, the k x k upper triangle R (column-major, column j holds rows 0..j), the
// right-hand side g (k + 1 entries, the last the residual outside the Krylov space) and a list
// of radii; prints, per radius, |y|, the predicted residual and y.
#include <cstdio>
#include <vector>

#include "hookstep.h"

int main() {
  int k = 0, nd = 0;
  if (std::scanf("%d %d", &k, &nd) != 2 || k <= 0 || nd <= 0) return 1;
  const int LD = k + 2;
  std::vector<double> R((size_t)LD * (k + 1), 0.0), g(k + 2, 0.0);
  for (int j = 0; j < k; ++j)
    for (int i = 0; i <= j; ++i)
      if (std::scanf("%lf", &R[(size_t)j * LD + i]) != 1) return 1;
  for (int i = 0; i <= k; ++i)
    if (std::scanf("%lf", &g[i]) != 1) return 1;
  Hookstep hs;
  hs.init(R.data(), LD, k, g.data());
  for (int t = 0; t < nd; ++t) {
    double delta = 0, pred = 0, ylen = 0;
    if (std::scanf("%lf", &delta) != 1) return 1;
    const std::vector<double> y = hs.solve(delta, &pred, &ylen);
    std::printf("%.17g %.17g\n", ylen, pred);
    for (int i = 0; i < k; ++i) std::printf("%.17g\n", y[i]);
  }
  return 0;
}
