// Host-side check of the FP64 <-> double-float conversions (compiled for the CPU by nvcc; no device
// code runs).  Reads doubles from stdin (one per line, as hex bit patterns); writes, per value, the
// bit patterns of hi and lo of df_from_double(d) and of df_to_double of that pair.
#include <cstdio>
#include <cstring>

#include "dfloat.cuh"

using namespace flups;

int main() {
  unsigned long long u;
  while (std::scanf("%llx", &u) == 1) {
    double d;
    std::memcpy(&d, &u, 8);
    const dfloat x = df_from_double(d);
    const double back = df_to_double(x);
    unsigned hb, lb;
    unsigned long long db;
    std::memcpy(&hb, &x.hi, 4);
    std::memcpy(&lb, &x.lo, 4);
    std::memcpy(&db, &back, 8);
    std::printf("%08x %08x %016llx\n", hb, lb, db);
  }
  return 0;
}
