// Onesweep pass kernels with 11-bit digits (three passes over 32-bit keys:
// 11 + 11 + 10 bits).
#include "onesweep.cuh"

namespace rs {

using S32 = uint32_t;
using S64 = unsigned long long;

// Tile shapes: index 0 is the default.  MINB is the number of resident
// blocks per SM the register budget is sized for.
static const OnesweepKernel kR11[] = {
    make_onesweep<11, 512, 16, false, S32, 2>(), make_onesweep<11, 512, 16, true, S32, 2>(),
    make_onesweep<11, 512, 16, false, S64, 2>(), make_onesweep<11, 512, 16, true, S64, 2>(),
    make_onesweep<11, 256, 32, false, S32, 2>(), make_onesweep<11, 256, 32, true, S32, 2>(),
    make_onesweep<11, 1024, 8, false, S32, 1>(), make_onesweep<11, 1024, 8, true, S32, 1>(),
};

const OnesweepKernel* onesweep_kernels_r11(int* count) {
  *count = int(sizeof(kR11) / sizeof(kR11[0]));
  return kR11;
}

}  // namespace rs
