// Fused simulation-step kernels for +-J couplings (all lattice degrees,
// shared-memory and wide layouts, with and without dilution).
#define ICM_PART 1
#include "pt_icm.cu"
