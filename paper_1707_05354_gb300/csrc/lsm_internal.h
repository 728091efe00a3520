// Hooks of the plain dictionary (lsm_api.cu) used by the serving engine
// (lsm_serve.cu): C++ only, not part of the C ABI.
#pragma once

#include "gpulsm.h"
#include "lsm_kernels.h"

namespace gpulsm {

// Sorted-batch buffers of a plain dictionary.  A batch is sorted into the
// next free buffer while earlier folds still read theirs, so the sorts of a
// run of inserts can get ahead of the folds by up to kBatchBufs - 2 batches
// (one buffer may hold level 0).
constexpr int kBatchBufs = 6;

// Full levels of the dictionary, newest first (the host's view of r).
LevelSet dict_levels(lsm_t* h);
// Makes `st` wait for the folds in flight on the handle's internal stream.
cudaError_t dict_join(lsm_t* h, cudaStream_t st);
// Ordered update batch (lsm_update_batch_ordered) without the argument
// checks; with checked = false the host does not wait for the key check
// (the caller guarantees keys < 2^31 - 1).
lsm_status dict_update_ordered(lsm_t* h, const uint32_t* keys, const uint32_t* vals, const uint8_t* del,
                               uint64_t n, cudaStream_t st, bool checked);
// Records `ev` once everything enqueued so far on `st` for this handle,
// including the fold it started on its internal stream, has run.
cudaError_t dict_record_applied(lsm_t* h, cudaEvent_t ev, cudaStream_t st);
uint64_t dict_r(const lsm_t* h);
uint32_t dict_L(const lsm_t* h);
uint32_t* dict_status_word(lsm_t* h);

}  // namespace gpulsm
