// Patch-kernel tilings of 64^2 patches (FP32 and FP64): one translation unit per
// patch size, so that the instantiations compile in parallel.
#include "patch_kernels.cuh"

namespace mlsd {

int patch_variants_n64(int precision, std::vector<PatchVariant> &out)
{
    if (precision == MLSD_FP32) {
        add_variant<64, 4, 8, float>(out);
        add_variant<64, 4, 8, float, 3>(out);
        add_variant<64, 4, 8, float, 3, 1, 1>(out);
        add_variant<64, 4, 8, float, 3, 1, 4>(out);
        add_variant<64, 4, 8, float, 2, 1, 4>(out);
        add_variant<64, 4, 4, float, 1, 1, 4>(out);
        add_variant<64, 4, 4, float, 2, 1, 4>(out);
        add_variant<64, 4, 4, float, 2, 1, 1>(out);
        add_variant<64, 4, 4, float>(out);
        add_variant<64, 2, 8, float>(out);
        add_variant<64, 8, 4, float>(out);
        add_variant<64, 2, 4, float>(out);
        add_variant2<64, 4, 4>(out);
        add_variant2<64, 2, 4>(out);
        add_variant2<64, 4, 2>(out);
        add_variant_tm<64, 4>(out);                     // coefficients in tensor memory
        add_variant_tm<64, 4, 1, 0, true>(out);         // ... column halos as the rows need them
    } else {
        add_variant<64, 2, 4, double>(out);
        add_variant<64, 4, 4, double>(out);
    }
    return (int)out.size();
}

}  // namespace mlsd
