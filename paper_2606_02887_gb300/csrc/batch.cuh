// Uneven batch engine (SNMF_DENSE_BATCH handles); defined in batch.cu.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/snmf.h"

namespace snmf {

struct BatchCtx;

// Argument checks only (no device work): SNMF_ERR_ARG with *err set, or SNMF_OK.
snmf_status batch_validate(const snmf_matrix* A, const snmf_options& opt, std::string* err);
// Validates the batch description, builds the work lists, converts and stores the
// problems' A (FP64 / FP32 / BF16, rows packed, columns padded to a common pitch) and
// computes ||A_p||_F^2 of the stored values.  On error returns the status and sets *err.
snmf_status batch_create(BatchCtx** out, const snmf_matrix* A, const snmf_options& opt, cudaStream_t s,
                         std::string* err);
// Solves every problem from W (and Ht; NULL: Ht = W; W NULL: Philox init per problem),
// in place; host == true: W / Ht are host buffers copied inside the call.
snmf_status batch_solve(BatchCtx* b, bool host, void* W, void* Ht, snmf_stats* out, std::string* err);
// Per-problem results of the last solve (arrays of nprob entries, any may be NULL).
snmf_status batch_problem_stats(BatchCtx* b, double* f, double* residual, double* pg_rel, int32_t* iters,
                                std::string* err);
snmf_status batch_get_factors(BatchCtx* b, void* W, void* Ht, std::string* err);
int batch_nprob(const BatchCtx* b);
// Budget (clock64 cycles) of the bounded device waits of the engine's tensor-core product.
void batch_set_budget(BatchCtx* b, long long cycles);
// Mean time (ms, CUDA events on the engine's stream) of one grouped A_p X_p product over
// every problem.
snmf_status batch_profile_ax(BatchCtx* b, int iters, double* ms, std::string* err);
void batch_destroy(BatchCtx* b);

}  // namespace snmf
