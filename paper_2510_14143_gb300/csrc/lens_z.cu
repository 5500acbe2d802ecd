// All-lengths Z pass of the batched path.
#include "lens.cuh"

namespace cubic {

cudaError_t launch_z_lens(int c, const LensTable<ZArgs> *tab, int64_t blocks, int mode, cudaStream_t st)
{
    return lens_for_class(c, [&](auto lens) {
        return lens_launch(k_zpass_lens<decltype(lens)>, lens_col_smem(lens), blocks, st, tab, mode);
    });
}

}  // namespace cubic
