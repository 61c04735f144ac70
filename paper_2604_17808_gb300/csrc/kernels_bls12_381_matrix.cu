// BLS12-381 scalar field: the matrix-form (tensor-core) pass kernels.
#define NTT_FIELD FieldBls12381Fr
#define NTT_NS bls12_381
#define NTT_PART_MATRIX
#include "ntt_kernels.inl"
