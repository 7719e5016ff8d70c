// Hop-kernel instantiations, F64 storage.
#define BRIDGE_PREC P_F64
#include "dslash_inst.inc"
