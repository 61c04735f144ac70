// BN254 scalar field: pass kernels of the 2^10-element tile.
#define NTT_FIELD FieldBn254Fr
#define NTT_NS bn254
#define NTT_PART_PASS 10
#include "ntt_kernels.inl"
