// Hop-kernel instantiations, F32 storage.
#define BRIDGE_PREC P_F32
#include "dslash_inst.inc"
