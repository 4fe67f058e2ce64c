// Stream-ordered device memory for handles and workspaces.
//
// cudaFree of a cudaMalloc allocation waits for every stream of the device,
// so a build or an hps_free in one thread stalled the solves running on
// other streams (the request server runs both at once).  All library
// allocations that live with a handle or a build therefore come from one
// memory pool per device through cudaMallocFromPoolAsync / cudaFreeAsync:
// an allocation is ordered on the stream that makes it, a free on the
// stream that last used the memory, and neither waits for other streams.
// The pool keeps no freed memory beyond its release threshold (0): what a
// free returns goes back to the device at the stream's next synchronisation
// point, so other allocators in the process see it as free again.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace hps {

// Allocate `bytes` on the current device, ordered on stream `st`: usable on
// `st` at once and on other streams once they are ordered after `st`.
cudaError_t dev_malloc(void** p, size_t bytes, cudaStream_t st);
// Free memory from dev_malloc, ordered on stream `st` (every use of it must
// be ordered before this point on `st`).
void dev_free(void* p, cudaStream_t st);
// Free memory from dev_malloc that no queued or running work uses any more
// (the caller has waited for it), on a library-owned non-blocking stream of
// the current device, so that the free orders after nothing else.
void dev_free_idle(void* p);
// Bytes the current device's pool holds beyond what is allocated from it
// (freed memory not yet given back): free memory for planning purposes.
size_t dev_pool_idle_bytes();

}  // namespace hps
