// Host-side check of the shared-memory FFT stages (the exact device code paths,
// executed stage by stage on the CPU): DIT with digit-reversed input and DIF with
// natural input against a direct O(n^2) DFT.  Prints one line per size:
//   n  max|DIT - DFT|/max|DFT|  max|DIF - DFT|/max|DFT|   (double), then the float errors.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1406_4350_gb300/csrc/fft_core.cuh"

using namespace chebfi;

template <typename R>
static void run(int n, int nlines, double* err_dit, double* err_dif) {
  using C = cplx<R>;
  std::vector<int> rad;
  if (!factor_radices(n, rad)) { printf("bad n %d\n", n); exit(1); }
  std::vector<int> rev = digit_reversal(n, rad);
  std::vector<C> tw(n);
  for (int k = 0; k < n; ++k) {
    double a = 2.0 * M_PI * (double)k / (double)n;
    tw[k] = cmake<C>(std::cos(a), -std::sin(a));
  }
  FFTPlan<R> pl;
  pl.n = n;
  pl.nst = (int)rad.size();
  for (int i = 0; i < pl.nst; ++i) pl.radix[i] = rad[i];
  pl.tw = tw.data();
  // lines laid out with an odd pitch and element stride 1
  const int pitch = n + 1;
  std::vector<double> xr(n * nlines), xi(n * nlines);
  srand(12345 + n);
  for (auto& v : xr) v = rand() / (double)RAND_MAX - 0.5;
  for (auto& v : xi) v = rand() / (double)RAND_MAX - 0.5;
  double e1 = 0, e2 = 0;
  for (int sign = -1; sign <= 1; sign += 2) {
    std::vector<C> a(pitch * nlines), b(pitch * nlines);
    for (int l = 0; l < nlines; ++l)
      for (int i = 0; i < n; ++i) {
        a[l * pitch + rev[i]] = cmake<C>(xr[l * n + i], xi[l * n + i]);  // DIT input: reversed
        b[l * pitch + i] = cmake<C>(xr[l * n + i], xi[l * n + i]);       // DIF input: natural
      }
    LineMap lm;
    lm.stride = pitch;
    const int nthr = 37;  // any thread count must give the same result
    for (int s = 0; s < pl.nst; ++s)
      for (int t = 0; t < nthr; ++t)
        sign < 0 ? dit_stage<-1, R>(a.data(), nlines, lm, 1, pl, s, t, nthr)
                 : dit_stage<1, R>(a.data(), nlines, lm, 1, pl, s, t, nthr);
    for (int s = pl.nst - 1; s >= 0; --s)
      for (int t = 0; t < nthr; ++t)
        sign < 0 ? dif_stage<-1, R>(b.data(), nlines, lm, 1, pl, s, t, nthr)
                 : dif_stage<1, R>(b.data(), nlines, lm, 1, pl, s, t, nthr);
    for (int l = 0; l < nlines; ++l) {
      double mx = 0, d1 = 0, d2 = 0;
      for (int k = 0; k < n; ++k) {
        long double sr = 0, si = 0;
        for (int j = 0; j < n; ++j) {
          long double ang = sign * 2.0L * M_PI * (long double)((long long)j * k % n) / n;
          sr += xr[l * n + j] * cosl(ang) - xi[l * n + j] * sinl(ang);
          si += xr[l * n + j] * sinl(ang) + xi[l * n + j] * cosl(ang);
        }
        mx = std::fmax(mx, std::hypot((double)sr, (double)si));
        C u = a[l * pitch + k];
        C v = b[l * pitch + rev[k]];
        d1 = std::fmax(d1, std::hypot((double)u.x - (double)sr, (double)u.y - (double)si));
        d2 = std::fmax(d2, std::hypot((double)v.x - (double)sr, (double)v.y - (double)si));
      }
      e1 = std::fmax(e1, d1 / mx);
      e2 = std::fmax(e2, d2 / mx);
    }
  }
  *err_dit = e1;
  *err_dif = e2;
}

int main() {
  const int sizes[] = {1, 2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 24, 25, 27, 30, 32, 45, 48, 60, 64, 75, 96, 100, 120, 128, 144, 160, 180, 192, 240, 250, 256};
  for (int n : sizes) {
    double a, b, c, d;
    run<double>(n, 5, &a, &b);
    run<float>(n, 5, &c, &d);
    printf("%d %.3e %.3e %.3e %.3e\n", n, a, b, c, d);
  }
  return 0;
}
