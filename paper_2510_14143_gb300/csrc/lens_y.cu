// All-lengths Y pass of the batched path.
#include "lens.cuh"

namespace cubic {

cudaError_t launch_x_lens(int c, int mode, const LensTable<XArgs> *tab, int64_t blocks, cudaStream_t st)
{
    switch (mode) {
    case XM_FWD: return launch_x_lens_mode<XM_FWD>(c, tab, blocks, st);
    case XM_RATIO: return launch_x_lens_mode<XM_RATIO>(c, tab, blocks, st);
    case XM_UPDATE: return launch_x_lens_mode<XM_UPDATE>(c, tab, blocks, st);
    case XM_FINAL: return launch_x_lens_mode<XM_FINAL>(c, tab, blocks, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_y_lens(int c, const LensTable<YArgs> *tab, int64_t blocks, int inverse, cudaStream_t st)
{
    return lens_for_class(c, [&](auto lens) {
        return lens_launch(k_ypass_lens<decltype(lens)>, lens_col_smem(lens), blocks, st, tab, inverse);
    });
}

}  // namespace cubic
