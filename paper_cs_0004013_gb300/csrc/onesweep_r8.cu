// Onesweep pass kernels with 8-bit digits (four passes over 32-bit keys).
#include "onesweep.cuh"
#include "onesweep_pipe.cuh"

namespace rs {

using S32 = uint32_t;
using S64 = unsigned long long;

// Shape 0 is the default.  MINB = resident blocks per SM the register budget
// is sized for; the last flag puts the lookback before the staging step.
static const OnesweepKernel kR8[] = {
    make_onesweep<8, 512, 16, false, S32, 2, false>(0), make_onesweep<8, 512, 16, true, S32, 2, false>(0),
    make_onesweep<8, 512, 16, false, S64, 2, false>(0), make_onesweep<8, 512, 16, true, S64, 2, false>(0),
    // two payload words (64-bit keys with a value: the other key word and the value),
    // with the interleaved 64-bit reads and writes of the 64-bit sorts
    make_onesweep<8, 512, 16, 2, S32, 2, false, true>(0), make_onesweep<8, 512, 16, 2, S64, 2, false, true>(0),
    // the interleaved variants of the default key+payload kernel (64-bit keys)
    make_onesweep<8, 512, 16, true, S32, 2, false, true>(0), make_onesweep<8, 512, 16, true, S64, 2, false, true>(0),
    make_onesweep<8, 512, 16, false, S32, 2, true>(1),  make_onesweep<8, 512, 16, true, S32, 2, true>(1),
    make_onesweep<8, 512, 24, false, S32, 2, false>(2), make_onesweep<8, 512, 24, true, S32, 2, false>(2),
    make_onesweep<8, 512, 24, false, S64, 2, false>(2),
    make_onesweep<8, 512, 24, true, S32, 2, false, true>(2),  // interleaved: 64-bit keys
    make_onesweep<8, 1024, 16, false, S32, 1, false>(3), make_onesweep<8, 1024, 16, true, S32, 1, false>(3),
    make_onesweep<8, 384, 20, false, S32, 2, false>(4), make_onesweep<8, 384, 20, true, S32, 2, false>(4),
    // persistent, software-pipelined (onesweep_pipe.cuh)
    make_onesweep_pipe<8, 512, 16, false, S32, 2>(5),   make_onesweep_pipe<8, 512, 16, true, S32, 1>(5),
    make_onesweep_pipe<8, 256, 24, false, S32, 3>(6),   make_onesweep_pipe<8, 256, 24, true, S32, 2>(6),
    make_onesweep_pipe<8, 384, 20, false, S32, 2>(7),   make_onesweep_pipe<8, 384, 20, true, S32, 1>(7),
    make_onesweep_pipe<8, 512, 24, false, S32, 1>(8),   make_onesweep_pipe<8, 512, 24, true, S32, 1>(8),
    make_onesweep_pipe<8, 256, 16, false, S32, 4>(9),   make_onesweep_pipe<8, 256, 16, true, S32, 2>(9),
    // smaller blocks, more of them per SM
    make_onesweep<8, 256, 24, false, S32, 4, false>(10), make_onesweep<8, 256, 24, true, S32, 3, false>(10),
    make_onesweep<8, 256, 32, false, S32, 3, false>(11), make_onesweep<8, 256, 32, true, S32, 2, false>(11),
    make_onesweep<8, 384, 24, false, S32, 2, false>(12), make_onesweep<8, 384, 24, true, S32, 2, false>(12),
};

const OnesweepKernel* onesweep_kernels_r8(int* count) {
  *count = int(sizeof(kR8) / sizeof(kR8[0]));
  return kR8;
}

}  // namespace rs
