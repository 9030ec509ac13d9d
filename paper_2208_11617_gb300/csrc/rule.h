// rule.h -- the automaton rule as passed to the kernels (host and device).
#pragma once

#include <stdint.h>

namespace sx {

// Per-step rule for the byte-sliced automaton: for each value s of
// (live neighbours + own state), whether a dead / a live cell ends alive.
// Built on the host from the birth/survive masks; only values that can turn
// a cell on are listed.
struct Rule {
    // Nonzero when the rule is "born with k, survive with k-1 or k" for an odd
    // k (B3/S23, B5/S45): then a cell is alive next iff (live neighbours | own
    // state) == k.  Holds k replicated in the 4 bytes of a word.
    uint32_t or_k;
    int32_t nk;
    uint32_t kbytes[28];  // s replicated in the 4 bytes of a word
    uint32_t bsel[28];    // all-ones if a dead cell with s live neighbours is born
    uint32_t ssel[28];    // all-ones if a live cell with s - 1 live neighbours survives
};

}  // namespace sx
