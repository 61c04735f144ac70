// BN254 scalar field: table generators, element-wise kernels and the field's
// launcher table.
#define NTT_FIELD FieldBn254Fr
#define NTT_NS bn254
#define NTT_PART_MISC
#include "ntt_kernels.inl"
