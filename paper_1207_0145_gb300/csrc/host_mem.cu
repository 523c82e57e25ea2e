// host_mem.cu -- page-locked host memory for mpsm_join_host's inputs (include/mpsm.h).
//
// A host-buffer join is bound by the host-to-device link.  Measured on Grace hosts, the
// link reads a page-locked buffer at its full rate (about 211 GB/s) where the buffer sits
// on huge pages; a plain page-locked allocation made once other processes had pinned and
// released many gigabytes held regions on base pages that copied at 10-100 GB/s.  These
// buffers are anonymous mappings on transparent huge pages, registered with the CUDA
// driver.  A buffer should be filled before the next large one is made: a kernel that
// splits underused huge pages splits those still holding only zeros when memory runs
// short.  The paper has no counterpart: its inputs start in memory.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
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

namespace {

// The size of a transparent huge page (the kernel's PMD mapping size: 2 MiB under 4 KiB base
// pages, 512 MiB under 64 KiB ones); 2 MiB where the kernel does not say.
uint64_t huge_page_bytes() {
  static uint64_t hp = 0;
  if (!hp) {
    unsigned long long v = 0;
    if (FILE* f = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
      if (fscanf(f, "%llu", &v) != 1) v = 0;
      fclose(f);
    }
    hp = (v >= 4096 && !(v & (v - 1))) ? (uint64_t)v : (2ull << 20);
  }
  return hp;
}

// The mapping behind `bytes`: whole huge pages from a buffer of one huge page up (a huge
// page covers only an aligned range the mapping holds whole), else the bytes themselves.
uint64_t mapped_bytes(uint64_t bytes) {
  const uint64_t hp = huge_page_bytes();
  return bytes >= hp ? (bytes + hp - 1) / hp * hp : bytes;
}

// One mapping of `len` bytes (from an aligned start when `whole`), advised for huge pages,
// populated and collapsed; nullptr where the mapping fails.
char* map_huge(uint64_t len, bool whole) {
  const uint64_t hp = huge_page_bytes();
  const uint64_t span = whole ? len + hp : len;
  void* raw = mmap(nullptr, span, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (raw == MAP_FAILED) return nullptr;
  char* p = static_cast<char*>(raw);
  if (whole) {  // give back the unaligned head and the tail
    const uint64_t head = (hp - (uint64_t)(uintptr_t)raw % hp) % hp;
    if (head) munmap(raw, head);
    munmap(p + head + len, hp - head);  // head < hp: the tail is never empty
    p += head;
  }
  // advice only, each step ignored where the kernel lacks it: huge pages for the mapping,
  // every page faulted in now, then ranges that got base pages collapsed into huge ones
  madvise(p, len, MADV_HUGEPAGE);
  madvise(p, len, MADV_POPULATE_WRITE);
  madvise(p, len, MADV_COLLAPSE);
  return p;
}

}  // namespace

MPSM_API int mpsm_host_alloc(uint64_t bytes, void** out) {
  if (!out || bytes == 0) return MPSM_ERR_INVALID_ARG;
  *out = nullptr;
  const uint64_t len = mapped_bytes(bytes);
  char* p = map_huge(len, bytes >= huge_page_bytes());
  if (!p) return MPSM_ERR_OOM;
  if (cudaHostRegister(p, len, cudaHostRegisterDefault) != cudaSuccess) {
    cudaGetLastError();
    munmap(p, len);
    return MPSM_ERR_CUDA;
  }
  *out = p;
  return MPSM_OK;
}

MPSM_API int mpsm_host_free(void* p, uint64_t bytes) {
  if (!p) return MPSM_OK;
  const cudaError_t e = cudaHostUnregister(p);
  munmap(p, mapped_bytes(bytes));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MPSM_ERR_CUDA;
  }
  return MPSM_OK;
}
