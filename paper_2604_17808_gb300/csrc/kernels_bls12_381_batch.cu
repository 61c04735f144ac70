// BLS12-381 scalar field: the persistent batched kernel.
#define NTT_FIELD FieldBls12381Fr
#define NTT_NS bls12_381
#define NTT_PART_BATCH
#include "ntt_kernels.inl"
