// Hop-kernel instantiations, F64 storage.
#define BRIDGE_PREC P_F64
#define BRIDGE_PREC_ID 0
#include "dslash_inst.inc"
