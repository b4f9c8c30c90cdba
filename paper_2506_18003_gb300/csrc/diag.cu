// Diagnostics: test-time fault injection (SCD_FAULT_INJECT) and NVTX ranges around the
// entry points.  Nothing here touches the GPU.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace scd {

bool fault_host(const char* site) {
  const char* v = getenv("SCD_FAULT_INJECT");
  if (!v || strncmp(v, "host:", 5) != 0 || strcmp(v + 5, site) != 0) return false;
  char msg[96];
  snprintf(msg, sizeof msg, "injected fault at %s", site);
  set_last_error(msg);
  return true;
}

int fault_batch_drop() {
  const char* v = getenv("SCD_FAULT_INJECT");
  if (!v || strncmp(v, "batch_drop:", 11) != 0) return -1;
  const int t = atoi(v + 11);
  return t >= 0 ? t : -1;
}

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

}  // namespace scd
