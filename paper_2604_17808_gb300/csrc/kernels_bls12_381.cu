// Kernels of the BLS12-381 scalar field.
#define NTT_FIELD FieldBls12381Fr
#include "ntt_kernels.inl"

namespace gb300ntt {
const FieldLaunchers &launchers_bls12_381() { return kLaunchers; }
}  // namespace gb300ntt
