// Patch-kernel tilings of 128^2 and 256^2 patches: each field split over a
// thread-block cluster, or a 128^2 field in one CTA with its coefficients in
// tensor memory (FP32).  A translation unit of its own, so that the
// instantiations compile in parallel with the others.
#include "patch_kernels.cuh"

namespace mlsd {

int patch_variants_cluster(int n, std::vector<PatchVariant> &out)
{
    if (n == 128) {
        add_variant<128, 4, 8, float, 3, 4>(out);
        add_variant<128, 4, 8, float, 3, 4, 1>(out);
        add_variant<128, 4, 8, float, 3, 4, 2>(out);
        add_variant<128, 4, 8, float, 3, 4, 3>(out);
        add_variant<128, 4, 4, float, 1, 4, 3>(out);
        add_variant<128, 4, 8, float, 1, 2>(out);
        add_variant<128, 4, 4, float, 1, 4>(out);
        add_variant<128, 2, 8, float, 2, 4, 3>(out);      // 2x8 cells: 16 warps per SM
        add_variant<128, 2, 8, float, 2, 4>(out);
        add_variant<128, 4, 8, float, 3, 4, 5>(out);      // bulk copies, cross-slab rows last
        add_variant<128, 4, 8, float, 2, 4, 5>(out);
        // coefficients in tensor memory: a whole field per CTA of 512 threads, or
        // clusters of 2 at 2 CTAs per SM
        add_variant_tm<128>(out);
        add_variant_tm<128, 2, 2, 3>(out);
        add_variant_tm<128, 1, 1, 0, true>(out);          // column halos as the rows need them
        add_variant_tm<128, 2, 2, 3, true>(out);
    } else if (n == 256) {
        add_variant<256, 4, 8, float, 1, 8>(out);
        add_variant<256, 4, 8, float, 1, 8, 1>(out);
        add_variant<256, 4, 8, float, 2, 8, 1>(out);
        add_variant<256, 4, 8, float, 1, 8, 2>(out);
        add_variant<256, 4, 8, float, 2, 8, 2>(out);
        add_variant<256, 4, 8, float, 3, 16, 2>(out);
        add_variant<256, 4, 8, float, 1, 8, 3>(out);
        add_variant<256, 4, 8, float, 3, 16, 3>(out);
        add_variant<256, 4, 4, float, 1, 8, 3>(out);
        add_variant<256, 4, 4, float, 1, 8>(out);
        add_variant<256, 4, 8, float, 3, 16>(out);
        add_variant<256, 2, 8, float, 1, 8, 3>(out);      // 2x8 cells: 16 warps per SM
        add_variant<256, 2, 8, float, 1, 8>(out);
        add_variant<256, 4, 8, float, 1, 8, 5>(out);      // bulk copies, cross-slab rows last
        add_variant<256, 4, 8, float, 3, 16, 5>(out);
        add_variant<256, 4, 8, float, 2, 16, 5>(out);
        add_variant<256, 2, 8, float, 1, 8, 5>(out);
        // coefficients in tensor memory: clusters of 4 CTAs of 512 threads, or of
        // 8 CTAs of 256 threads at 2 CTAs per SM
        add_variant_tm<256, 1, 4, 3>(out);
        add_variant_tm<256, 2, 8, 3>(out);
        add_variant_tm<256, 1, 4, 3, true>(out);          // column halos as the rows need them
        add_variant_tm<256, 2, 8, 3, true>(out);
    }
    return (int)out.size();
}

}  // namespace mlsd
