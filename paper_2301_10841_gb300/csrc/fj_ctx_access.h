// Internal accessors of a context for the library's other translation units.
#pragma once

#include <cuda_runtime.h>

#include "../../include/fj.h"

cudaStream_t fj_internal_ctx_stream(const fj_ctx* c);
int fj_internal_ctx_device(const fj_ctx* c);
// Device pointer of column `col` of a relation (NULL when out of range).
const int32_t* fj_internal_rel_col(const fj_rel* r, int col);
// Predictions of a model for n host rows of `dim` features, standardized
// with the model's scaler first; host output.  Synchronizes.
fj_status fj_internal_model_predict(fj_model* m, const float* host_x, int n, int dim,
                                    float* host_y);
