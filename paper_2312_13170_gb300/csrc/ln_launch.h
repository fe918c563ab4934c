// Host-side launch with programmatic stream serialisation (programmatic
// dependent launch): the kernel's CTAs may start while its predecessor in the
// stream is finishing; the kernel must execute griddepcontrol.wait (pdl_wait
// in ln_async.cuh) before its first access to memory the predecessor writes.
#pragma once

#include <cuda_runtime.h>

#include "ln_internal.h"

namespace ln {

template <class... KArgs, class... Args>
ln_status pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, const char *what,
                     Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
    if (e != cudaSuccess) return fail(LN_ERR_CUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return check_launch(what);
}

}  // namespace ln
