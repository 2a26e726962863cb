// Host-side text of a device status word (layout in common.cuh): the code in
// bits 60..63; for ABM_ERR_NONFINITE the trajectory (bits 32..59) and step
// (bits 0..31) of the first non-finite value; for ABM_ERR_TIMEOUT the site of
// the wait (bits 56..59), the unit that waited (32..55) and a position (0..31);
// for ABM_ERR_BOUNDS (checked build) the kernel (bits 52..59) and the index
// (bits 0..51).
#pragma once
#include <cstdio>

#include "../../include/abm.h"

namespace abm {

inline void status_text(unsigned long long w, char* buf, size_t len) {
  const int code = (int)(w >> 60);
  const unsigned long long pos = w & 0xFFFFFFFFull;
  if (code == ABM_ERR_NONFINITE) {
    std::snprintf(buf, len, "a non-finite value at trajectory %llu, step %llu", (w >> 32) & 0x0FFFFFFFull, pos);
    return;
  }
  if (code == ABM_ERR_BOUNDS) {
    const char* const kSites[] = {"?", "setup", "near", "split near", "FP64 far", "FP32 far",
                                         "per-component far", "tensor-core far", "single-trajectory",
                                         "history import", "history export", "adjoint", "weights"};
    const int site = (int)((w >> 52) & 0xFF);
    std::snprintf(buf, len, "an index outside its buffer in the %s kernel (index %llu); the access was skipped",
                  site < (int)(sizeof(kSites) / sizeof(kSites[0])) ? kSites[site] : "?", w & 0xFFFFFFFFFFFFFull);
    return;
  }
  if (code != ABM_ERR_TIMEOUT) {
    std::snprintf(buf, len, "status code %d (detail 0x%llx)", code, w & 0x0FFFFFFFFFFFFFFFull);
    return;
  }
  const int site = (int)((w >> 56) & 0xF);
  const unsigned long long idx = (w >> 32) & 0xFFFFFFull;
  switch (site) {
    case 1:
      std::snprintf(buf, len, "a wait that ran out: the stepping CTA waited for the far sums of time tile %llu", idx);
      break;
    case 2:
      std::snprintf(buf, len, "a wait that ran out: a far CTA waited for the history rows before time tile %llu",
                    idx);
      break;
    case 3:
      std::snprintf(buf, len, "a wait that ran out: the tensor-core far kernel's loader (column tile %llu) after %llu "
                    "loads", idx, pos);
      break;
    case 4:
      std::snprintf(buf, len, "a wait that ran out: the tensor-core far kernel's MMA issuer (column tile %llu) waited "
                    "for accumulator chunk %llu to drain", idx, pos);
      break;
    case 5:
      std::snprintf(buf, len, "a wait that ran out: the tensor-core far kernel's MMA issuer (column tile %llu) waited "
                    "for the operands of K block %llu", idx, pos);
      break;
    default:
      std::snprintf(buf, len, "a wait that ran out (site %d, unit %llu, position %llu)", site, idx, pos);
  }
}

}  // namespace abm
