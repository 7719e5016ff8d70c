// Hop-kernel instantiations, F16 storage.
#define BRIDGE_PREC P_F16
#include "dslash_inst.inc"
