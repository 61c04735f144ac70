// BLS12-381 scalar field: pass kernels of the 2^10-element tile.
#define NTT_FIELD FieldBls12381Fr
#define NTT_NS bls12_381
#define NTT_PART_PASS 10
#include "ntt_kernels.inl"
