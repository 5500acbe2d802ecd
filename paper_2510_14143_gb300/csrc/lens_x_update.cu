// All-lengths X pass of the batched path, mode XM_UPDATE.
#include "lens.cuh"

namespace cubic {
CUBIC_LENS_X_UNIT(XM_UPDATE)
}  // namespace cubic
