// Host-side check of the register DFTs of the FFT engine (compiled for the CPU by nvcc; no device
// code runs).  Reads, from stdin, lines "R inv zh n" followed by n complex inputs (re im); writes
// the R outputs of the engine's radix-R DFT (forward exp(-2 pi i q r / R), inverse the conjugate,
// unnormalised) in FP64, one "re im" pair per line.
#include <cstdio>

#include "fft_engine.cuh"

using namespace flups;

template <bool INV, bool ZH>
static void run(int R, double2* v) {
  switch (R) {
    case 2: dftR<double, 2, INV>(v); break;
    case 3: dftR<double, 3, INV>(v); break;
    case 4: dftR<double, 4, INV>(v); break;
    case 8: dftR<double, 8, INV>(v); break;
    case 16: dftR<double, 16, INV>(v); break;
    case 32: dft32<double, INV, ZH>(v); break;
    case 44: dft4_half<double, INV>(v[0], v[1], v[2], v[3]); break;  // DFT-4 of (a, b, 0, 0)
    default: break;
  }
}

int main() {
  int R, inv, zh, n;
  while (std::scanf("%d %d %d %d", &R, &inv, &zh, &n) == 4) {
    double2 v[32];
    for (int i = 0; i < n && i < 32; ++i) {
      if (std::scanf("%lf %lf", &v[i].x, &v[i].y) != 2) return 1;
    }
    if (inv) {
      if (zh) run<true, true>(R, v); else run<true, false>(R, v);
    } else {
      if (zh) run<false, true>(R, v); else run<false, false>(R, v);
    }
    const int m = R == 44 ? 4 : R;
    for (int i = 0; i < m; ++i) std::printf("%.17g %.17g\n", v[i].x, v[i].y);
  }
  return 0;
}
