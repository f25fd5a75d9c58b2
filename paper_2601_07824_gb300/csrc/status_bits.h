// status_bits.h -- bits a kernel may set in the context's device status word.
#pragma once
namespace hm {
enum : int { ST_TIMEOUT = 1, ST_BADARG = 2, ST_NONPOS = 4 };  // ST_NONPOS: S(a) + eps <= 0 (Algorithm 3)
// Default iteration limit of every bounded inter-CTA wait (hadamag_set_wait_limit changes a
// context's copy).
constexpr long long kDefaultSpinLimit = 1ll << 25;
}
