// Patch-kernel tilings of 32^2 patches (FP32 and FP64): one translation unit per
// patch size, so that the instantiations compile in parallel.
#include "patch_kernels.cuh"

namespace mlsd {

int patch_variants_n32(int precision, std::vector<PatchVariant> &out)
{
    if (precision == MLSD_FP32) {
        add_variant<32, 4, 8, float>(out);
        add_variant<32, 4, 8, float, 1, 1, 1>(out);
        add_variant<32, 4, 8, float, 1, 1, 4>(out);
        add_variant<32, 4, 4, float>(out);
        add_variant<32, 2, 8, float>(out);
        add_variant<32, 2, 4, float>(out);
        add_variant2<32, 4, 4>(out);
        add_variant2<32, 2, 4>(out);
        add_variant2<32, 4, 2>(out);
    } else {
        add_variant<32, 2, 4, double>(out);
        add_variant<32, 4, 4, double>(out);
    }
    return (int)out.size();
}

}  // namespace mlsd
