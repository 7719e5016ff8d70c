// Hop-kernel instantiations, BF16 storage.
#define BRIDGE_PREC P_BF16
#include "dslash_inst.inc"
