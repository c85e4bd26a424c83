// Fused GETT (algorithm 0): the whole contraction in one kernel.  FP64 and
// FP32 run the SIMT tiled form; the tensor-core dtypes run on tcgen05.
#include <cuda_runtime.h>

#include "tc_internal.h"

namespace tc {

tc_status exec_gett_simt(Plan &p, const void *alpha, const void *A, const void *B,
                         const void *beta, void *C, void *stream);

size_t gett_workspace_bytes(const Plan &) { return 0; }

void gett_release(Plan &) {}

tc_status exec_gett(Plan &p, const void *alpha, const void *A, const void *B,
                    const void *beta, void *C, void *stream) {
    if (p.dtype == TC_F64 || p.dtype == TC_F32)
        return exec_gett_simt(p, alpha, A, B, beta, C, stream);
    return fail(TC_ERROR_UNSUPPORTED_DTYPE, "tensor-core GETT not built yet");
}

}  // namespace tc
