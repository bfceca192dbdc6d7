// Host driver for the FP64 <-> FP32-pair conversions and df64 arithmetic of fpconv.cuh.
// stdin: lines "op x y" with x, y as 16-hex-digit FP64 bit patterns; stdout: result bits.
#include <cinttypes>
#include <cstdio>
#include <cstring>

#include "../../paper_2104_08863_gb300/csrc/fpconv.cuh"

using namespace pp;

int main() {
  char op[16];
  unsigned long long xb, yb;
  while (std::scanf("%15s %llx %llx", op, &xb, &yb) == 3) {
    const double x = double_of(xb), y = double_of(yb);
    if (!std::strcmp(op, "trunc")) {
      std::printf("%08x\n", bits_of(f64_to_f32_trunc(x)));
    } else if (!std::strcmp(op, "split")) {
      float hi, lo;
      f64_split(x, hi, lo);
      std::printf("%08x %08x\n", bits_of(hi), bits_of(lo));
    } else if (!std::strcmp(op, "sum")) {    // x, y carry FP32 values widened to FP64
      std::printf("%016llx\n", (unsigned long long)bits_of(f32_add_to_f64((float)x, (float)y)));
    } else if (!std::strcmp(op, "widen")) {  // x carries an FP32 value widened to FP64
      std::printf("%016llx\n", (unsigned long long)bits_of(f32_to_f64_exact((float)x)));
    } else if (!std::strcmp(op, "dfadd") || !std::strcmp(op, "dfmul")) {
      float xh, xl, yh, yl;
      f64_split(x, xh, xl);
      f64_split(y, yh, yl);
      const df r = !std::strcmp(op, "dfadd") ? df_add(df{xh, xl}, df{yh, yl}) : df_mul(df{xh, xl}, df{yh, yl});
      std::printf("%08x %08x\n", bits_of(r.hi), bits_of(r.lo));
    } else if (!std::strcmp(op, "twodiff")) {   // exact difference of two FP32 values
      const df r = two_diff_df((float)x, (float)y);
      std::printf("%08x %08x\n", bits_of(r.hi), bits_of(r.lo));
    }
  }
  return 0;
}
