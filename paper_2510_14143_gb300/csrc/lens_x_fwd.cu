// All-lengths X pass of the batched path, mode XM_FWD.
#include "lens.cuh"

namespace cubic {
CUBIC_LENS_X_UNIT(XM_FWD)
}  // namespace cubic
