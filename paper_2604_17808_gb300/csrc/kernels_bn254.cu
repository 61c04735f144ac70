// Kernels of the BN254 scalar field.
#define NTT_FIELD FieldBn254Fr
#include "ntt_kernels.inl"

namespace gb300ntt {
const FieldLaunchers &launchers_bn254() { return kLaunchers; }
}  // namespace gb300ntt
