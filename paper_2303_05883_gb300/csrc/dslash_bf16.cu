// Hop-kernel instantiations, BF16 storage.
#define BRIDGE_PREC P_BF16
#define BRIDGE_PREC_ID 3
#include "dslash_inst.inc"
