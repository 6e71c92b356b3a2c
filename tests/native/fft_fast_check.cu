// Host-side check of the two-pass line FFTs (the device code paths, run pass by pass on
// the CPU): F from natural order to split order and G from split order to natural order,
// both against a direct DFT, for every compiled length.  Prints: N errF errG (double) errF
// errG (float).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1406_4350_gb300/csrc/fft_fast.cuh"

using namespace chebfi;

template <int N, typename R>
static void run(double* eF, double* eG) {
  using C = cplx<R>;
  std::vector<C> tw(N);
  for (int k = 0; k < N; ++k) tw[k] = cmake<C>(std::cos(2 * M_PI * k / N), -std::sin(2 * M_PI * k / N));
  const int nlines = 7, pitch = N + 1, nthr = 29;
  LineMap lm;
  lm.stride = pitch;
  double e1 = 0, e2 = 0;
  for (int sign = -1; sign <= 1; sign += 2) {
    std::vector<double> xr(N * nlines), xi(N * nlines);
    srand(777 + N);
    for (auto& v : xr) v = rand() / (double)RAND_MAX - 0.5;
    for (auto& v : xi) v = rand() / (double)RAND_MAX - 0.5;
    std::vector<C> a(pitch * nlines), b(pitch * nlines);
    for (int l = 0; l < nlines; ++l)
      for (int i = 0; i < N; ++i) a[l * pitch + i] = cmake<C>(xr[l * N + i], xi[l * N + i]);
    // G's input: the same sequence placed in split order
    for (int l = 0; l < nlines; ++l)
      for (int p = 0; p < N; ++p) {
        const int k = fast::split_index<N>(p);
        b[l * pitch + p] = cmake<C>(xr[l * N + k], xi[l * N + k]);
      }
    for (int t = 0; t < nthr; ++t)
      sign < 0 ? fast::F_passA<N, -1>(a.data(), nlines, lm, 1, tw.data(), t, nthr)
               : fast::F_passA<N, 1>(a.data(), nlines, lm, 1, tw.data(), t, nthr);
    for (int t = 0; t < nthr; ++t)
      sign < 0 ? fast::F_passB<N, -1>(a.data(), nlines, lm, 1, t, nthr) : fast::F_passB<N, 1>(a.data(), nlines, lm, 1, t, nthr);
    for (int t = 0; t < nthr; ++t)
      sign < 0 ? fast::G_passB<N, -1>(b.data(), nlines, lm, 1, tw.data(), t, nthr)
               : fast::G_passB<N, 1>(b.data(), nlines, lm, 1, tw.data(), t, nthr);
    for (int t = 0; t < nthr; ++t)
      sign < 0 ? fast::G_passA<N, -1>(b.data(), nlines, lm, 1, t, nthr) : fast::G_passA<N, 1>(b.data(), nlines, lm, 1, t, nthr);
    for (int l = 0; l < nlines; ++l) {
      double mx = 0, d1 = 0, d2 = 0;
      for (int k = 0; k < N; ++k) {
        long double sr = 0, si = 0;
        for (int j = 0; j < N; ++j) {
          long double ang = sign * 2.0L * M_PI * (long double)((long long)j * k % N) / N;
          sr += xr[l * N + j] * cosl(ang) - xi[l * N + j] * sinl(ang);
          si += xr[l * N + j] * sinl(ang) + xi[l * N + j] * cosl(ang);
        }
        mx = std::fmax(mx, std::hypot((double)sr, (double)si));
        // F: X[k] sits at the position p with split_index(p) = k
        int p = 0;
        while (fast::split_index<N>(p) != k) ++p;
        const C u = a[l * pitch + p];
        d1 = std::fmax(d1, std::hypot((double)u.x - (double)sr, (double)u.y - (double)si));
        const C v = b[l * pitch + k];
        d2 = std::fmax(d2, std::hypot((double)v.x - (double)sr, (double)v.y - (double)si));
      }
      e1 = std::fmax(e1, d1 / mx);
      e2 = std::fmax(e2, d2 / mx);
    }
  }
  *eF = e1;
  *eG = e2;
}

template <int N> static void row() {
  double a, b, c, d;
  run<N, double>(&a, &b);
  run<N, float>(&c, &d);
  printf("%d %.3e %.3e %.3e %.3e\n", N, a, b, c, d);
}

int main() {
  row<16>(); row<24>(); row<32>(); row<48>(); row<64>(); row<72>(); row<96>(); row<120>(); row<128>(); row<144>();
  return 0;
}
