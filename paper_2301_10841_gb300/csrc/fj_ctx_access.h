// Internal accessors of a context for the library's other translation units.
#pragma once

#include <cuda_runtime.h>

#include "../../include/fj.h"

cudaStream_t fj_internal_ctx_stream(const fj_ctx* c);
int fj_internal_ctx_device(const fj_ctx* c);
