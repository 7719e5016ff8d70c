// Hop-kernel instantiations, F32 storage.
#define BRIDGE_PREC P_F32
#define BRIDGE_PREC_ID 1
#include "dslash_inst.inc"
