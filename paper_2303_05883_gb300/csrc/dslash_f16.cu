// Hop-kernel instantiations, F16 storage.
#define BRIDGE_PREC P_F16
#define BRIDGE_PREC_ID 2
#include "dslash_inst.inc"
