// BN254 scalar field: the matrix-form (tensor-core) pass kernels.
#define NTT_FIELD FieldBn254Fr
#define NTT_NS bn254
#define NTT_PART_MATRIX
#include "ntt_kernels.inl"
