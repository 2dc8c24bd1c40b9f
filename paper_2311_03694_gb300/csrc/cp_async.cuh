// 16-byte asynchronous global -> shared copies (cp.async, sm_80 and later):
// the copy (both addresses 16-byte aligned), its commit group, and the wait
// until at most N groups of this thread are still in flight.
#pragma once

#include <stdint.h>

#include "ptx.cuh"

namespace grom {
namespace ptx {

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace ptx
}  // namespace grom
