// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ba.h"

namespace ba {

// Launch accounting (ba_kernel_launch_count).
void count_launch(uint64_t n = 1);

// Record a message for ba_last_error() and return st.
ba_status set_error(ba_status st, const char* fmt, ...);

// Stable radix sort + row pointers (ba_sort.cu).  scratch must hold
// csr_scratch_bytes(n) bytes; d_err gets bit 0 set for a key outside
// [0, n_keys).
size_t csr_scratch_bytes(int n);
cudaError_t csr_build_async(const int32_t* keys, int n, int n_keys, int32_t* perm_out,
                            int32_t* rowptr_out, void* scratch, int* d_err, cudaStream_t s);

}  // namespace ba
