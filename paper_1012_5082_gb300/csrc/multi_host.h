// multi_host.h -- host-side access to a multicomponent object's state, for
// a binary context that runs its colour steps through a two-species
// multicomponent object (vcsgc_capi.cu).  Status codes as in vcsgc.h.
#pragma once

#include "multi.cuh"

namespace vcsgc {

// running state of replica r (the pending step applied first)
int multi_get_state(void* m, int r, MRepState* out);
// replace it (forms without a deferred commit only)
int multi_set_state(void* m, int r, const MRepState* in);
// densities rho_i of replica r (N doubles, host)
int multi_get_rho(void* m, int r, double* out);
// the object takes its local decisions on the FP32-screened dE
bool multi_screened(void* m);
// device species bytes of replica r (the pending step applied first), or
// null on an error
const uint8_t* multi_types_device(void* m, int r);

}  // namespace vcsgc
