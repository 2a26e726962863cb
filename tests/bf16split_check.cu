// Host-side check of the split-precision conversions in csrc/bf16split.cuh
// (compiled by tests/test_bf16split.py with nvcc for the host only).
//   bf16split_check split IN OUT : reads n doubles, writes per input the three
//                                  BF16 piece patterns (uint16 x 3) and a flag
//                                  per piece (1 = integer path)
//   bf16split_check f32          : every float bit pattern through
//                                  f32_bits_to_f64 against the host's
//                                  conversion; prints the mismatch count
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../paper_1611_08678_gb300/csrc/bf16split.cuh"

int main(int argc, char** argv) {
  if (argc >= 2 && !strcmp(argv[1], "f32")) {
    unsigned long long bad = 0;
    for (unsigned long long v = 0; v <= 0xFFFFFFFFull; ++v) {
      const uint32_t u = (uint32_t)v;
      float f;
      memcpy(&f, &u, 4);
      if (f != f) continue;  // NaN: any NaN will do, both sides convert by instruction
      const double want = (double)f;
      const double got = abm::f32_bits_to_f64(u);
      if (abm::f64_bits(want) != abm::f64_bits(got)) ++bad;
    }
    printf("%llu\n", bad);
    return 0;
  }
  if (argc >= 4 && !strcmp(argv[1], "split")) {
    FILE* in = fopen(argv[2], "rb");
    if (!in) return 2;
    std::vector<double> x;
    double v;
    while (fread(&v, 8, 1, in) == 1) x.push_back(v);
    fclose(in);
    FILE* out = fopen(argv[3], "wb");
    if (!out) return 2;
    for (double xi : x) {
      __nv_bfloat16 pcs[3];
      abm::split3_bf16(xi, pcs);
      uint16_t rec[6];
      double r = xi;
      for (int k = 0; k < 3; ++k) {
        __nv_bfloat16_raw raw = pcs[k];
        rec[k] = raw.x;
        uint16_t b;
        double p;
        rec[3 + k] = abm::bf16_round_int(r, b, p) ? 1 : 0;
        r -= (double)__bfloat162float(pcs[k]);
      }
      fwrite(rec, 2, 6, out);
    }
    fclose(out);
    return 0;
  }
  return 1;
}
