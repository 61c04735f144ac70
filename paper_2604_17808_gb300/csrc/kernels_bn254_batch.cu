// BN254 scalar field: the persistent batched kernel.
#define NTT_FIELD FieldBn254Fr
#define NTT_NS bn254
#define NTT_PART_BATCH
#include "ntt_kernels.inl"
