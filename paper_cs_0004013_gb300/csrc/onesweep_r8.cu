// Onesweep pass kernels with 8-bit digits (four passes over 32-bit keys).
#include "onesweep.cuh"
#include "onesweep2.cuh"

namespace rs {

using S32 = uint32_t;
using S64 = unsigned long long;

// Tile shapes (rs_plan.tile = shape + 1).  MINB = resident blocks per SM the
// register budget is sized for.
//   0: 512 x 16, lane-mask tables (onesweep.cuh): every payload layout, 64-bit
//      status words, the interleaved 64-bit reads and writes;
//   1: 384 x 24, half-warp rank groups (onesweep2.cuh), three blocks per SM:
//      the keys-only default above 2^22 keys;
//   2: 512 x 24, lane-mask tables: the key+payload default above 2^22 keys;
//   3: 1024 x 16, lane-mask tables, one block per SM;
//   4-6: half-warp rank groups at 512 x 24, 512 x 16 and 256 x 24;
//   7: 384 x 24, lane-mask tables, three blocks per SM: the key+payload
//      default above 2^21 keys (2^26: 322 us per pass against 332 at 512 x 24)
//      and, with interleaved words, the 64-bit keys default above 2^22 keys
//      (335 against 349 us); with two payload words it spills and gains nothing.
// GB300, 2^26 uniform 31-bit keys, per pass: shape 1 233 us (keys), shape 2
// 260 us (keys) and 343 us (key+payload), shape 4 238 / 385 us.
static const OnesweepKernel kR8[] = {
    make_onesweep<8, 512, 16, false, S32, 2, false>(0), make_onesweep<8, 512, 16, true, S32, 2, false>(0),
    make_onesweep<8, 512, 16, false, S64, 2, false>(0), make_onesweep<8, 512, 16, true, S64, 2, false>(0),
    // two payload words (64-bit keys with a value: the other key word and the value),
    // with the interleaved 64-bit reads and writes of the 64-bit sorts
    make_onesweep<8, 512, 16, 2, S32, 2, false, true>(0), make_onesweep<8, 512, 16, 2, S64, 2, false, true>(0),
    // the interleaved variants of the key+payload kernel (64-bit keys)
    make_onesweep<8, 512, 16, true, S32, 2, false, true>(0), make_onesweep<8, 512, 16, true, S64, 2, false, true>(0),
    make_onesweep2<384, 24, 0, S32, 3>(1), make_onesweep2<384, 24, 1, S32, 3>(1),
    make_onesweep2<384, 24, 0, S64, 3>(1), make_onesweep2<384, 24, 1, S64, 3>(1),
    make_onesweep<8, 512, 24, false, S32, 2, false>(2), make_onesweep<8, 512, 24, true, S32, 2, false>(2),
    make_onesweep<8, 512, 24, false, S64, 2, false>(2),
    make_onesweep<8, 512, 24, true, S32, 2, false, true>(2),  // interleaved: 64-bit keys
    make_onesweep<8, 1024, 16, false, S32, 1, false>(3), make_onesweep<8, 1024, 16, true, S32, 1, false>(3),
    make_onesweep2<512, 24, 0, S32, 2>(4), make_onesweep2<512, 24, 1, S32, 2>(4),
    make_onesweep2<512, 24, 0, S64, 2>(4), make_onesweep2<512, 24, 1, S64, 2>(4),
    make_onesweep2<512, 16, 0, S32, 2>(5), make_onesweep2<512, 16, 1, S32, 2>(5),
    make_onesweep2<256, 24, 0, S32, 4>(6), make_onesweep2<256, 24, 1, S32, 4>(6),
    make_onesweep<8, 384, 24, false, S32, 3, false>(7), make_onesweep<8, 384, 24, true, S32, 3, false>(7),
    make_onesweep<8, 384, 24, true, S32, 3, false, true>(7),  // interleaved: 64-bit keys
};

const OnesweepKernel* onesweep_kernels_r8(int* count) {
  *count = int(sizeof(kR8) / sizeof(kR8[0]));
  return kR8;
}

}  // namespace rs
