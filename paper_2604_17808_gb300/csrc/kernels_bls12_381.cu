// BLS12-381 scalar field: table generators, element-wise kernels and the field's
// launcher table.
#define NTT_FIELD FieldBls12381Fr
#define NTT_NS bls12_381
#define NTT_PART_MISC
#include "ntt_kernels.inl"
