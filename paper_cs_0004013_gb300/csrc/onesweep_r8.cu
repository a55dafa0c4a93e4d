// Onesweep pass kernels with 8-bit digits (four passes over 32-bit keys).
#include "onesweep.cuh"

namespace rs {

using S32 = uint32_t;
using S64 = unsigned long long;

static const OnesweepKernel kR8[] = {
    make_onesweep<8, 512, 16, false, S32, 2>(), make_onesweep<8, 512, 16, true, S32, 2>(),
    make_onesweep<8, 512, 16, false, S64, 2>(), make_onesweep<8, 512, 16, true, S64, 2>(),
    make_onesweep<8, 256, 32, false, S32, 2>(), make_onesweep<8, 256, 32, true, S32, 2>(),
    make_onesweep<8, 384, 20, false, S32, 2>(), make_onesweep<8, 384, 20, true, S32, 2>(),
};

const OnesweepKernel* onesweep_kernels_r8(int* count) {
  *count = int(sizeof(kR8) / sizeof(kR8[0]));
  return kR8;
}

}  // namespace rs
