// Fused simulation-step kernels for Gaussian couplings (all lattice degrees,
// shared-memory and wide layouts, with and without dilution).
#define ICM_PART 2
#include "pt_icm.cu"
