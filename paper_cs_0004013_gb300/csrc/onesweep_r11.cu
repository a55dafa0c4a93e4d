// Onesweep pass kernels with 11-bit digits (three passes over 32-bit keys:
// 11 + 11 + 10 bits).
#include "onesweep.cuh"

namespace rs {

using S32 = uint32_t;
using S64 = unsigned long long;

// Shape 0 is the default.  MINB = resident blocks per SM the register budget
// is sized for; the last flag puts the lookback before the staging step.
static const OnesweepKernel kR11[] = {
    make_onesweep<11, 1024, 16, false, S32, 1, false>(0), make_onesweep<11, 1024, 16, true, S32, 1, false>(0),
    make_onesweep<11, 1024, 16, false, S64, 1, false>(0), make_onesweep<11, 1024, 16, true, S64, 1, false>(0),
    make_onesweep<11, 1024, 16, false, S32, 1, true>(1),  make_onesweep<11, 1024, 16, true, S32, 1, true>(1),
    make_onesweep<11, 512, 16, false, S32, 2, false>(2),  make_onesweep<11, 512, 16, true, S32, 2, false>(2),
    make_onesweep<11, 1024, 24, false, S32, 1, false>(3), make_onesweep<11, 1024, 24, true, S32, 1, false>(3),
};

const OnesweepKernel* onesweep_kernels_r11(int* count) {
  *count = int(sizeof(kR11) / sizeof(kR11[0]));
  return kR11;
}

}  // namespace rs
