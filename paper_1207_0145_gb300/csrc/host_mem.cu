// host_mem.cu -- page-locked host memory for mpsm_join_host's inputs (include/mpsm.h).
//
// A host-buffer join is bound by the host-to-device link, and that link reads a
// page-locked buffer at its full rate only where the buffer's physical pages are
// contiguous enough for the device's address translation.  A plain page-locked
// allocation made once host memory is fragmented (after other processes pinned and
// released many gigabytes) can hold regions that copy at a tenth of the rate.  These
// buffers are anonymous mappings on transparent huge pages, registered with the CUDA
// driver.  The paper has no counterpart: its inputs start in memory.
#include <cuda_runtime.h>
#include <stdint.h>
#include <sys/mman.h>

#include "mpsm.h"

#define MPSM_API extern "C" __attribute__((visibility("default")))

// Linux madvise advice values (asm-generic), for headers that predate them
#ifndef MADV_POPULATE_WRITE
#define MADV_POPULATE_WRITE 23
#endif
#ifndef MADV_COLLAPSE
#define MADV_COLLAPSE 25
#endif

MPSM_API int mpsm_host_alloc(uint64_t bytes, void** out) {
  if (!out || bytes == 0) return MPSM_ERR_INVALID_ARG;
  *out = nullptr;
  void* p = mmap(nullptr, bytes, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (p == MAP_FAILED) return MPSM_ERR_OOM;
  // advice only, each step ignored where the kernel lacks it: huge pages for the mapping,
  // every page faulted in now, then ranges that got base pages collapsed into huge ones
  madvise(p, bytes, MADV_HUGEPAGE);
  madvise(p, bytes, MADV_POPULATE_WRITE);
  madvise(p, bytes, MADV_COLLAPSE);
  if (cudaHostRegister(p, bytes, cudaHostRegisterDefault) != cudaSuccess) {
    cudaGetLastError();
    munmap(p, bytes);
    return MPSM_ERR_CUDA;
  }
  *out = p;
  return MPSM_OK;
}

MPSM_API int mpsm_host_free(void* p, uint64_t bytes) {
  if (!p) return MPSM_OK;
  const cudaError_t e = cudaHostUnregister(p);
  munmap(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MPSM_ERR_CUDA;
  }
  return MPSM_OK;
}
