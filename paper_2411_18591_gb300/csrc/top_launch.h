// Kernel launch, dynamic shared memory and asynchronous-copy spellings used by every unit.
#pragma once

#ifndef TOP_LAUNCH
#define TOP_LAUNCH(kernel, grid, block, smem, stream, ...) kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__)
#endif

#ifndef TOP_DYN_SMEM
#define TOP_DYN_SMEM(T, name) extern __shared__ T name[]
#endif

#ifndef TOP_ASYNC_COPY
#define TOP_ASYNC_COPY
// 16-byte global -> shared copy that completes asynchronously (cached in L2 only); both addresses
// must be 16-byte aligned. top_cp_async_wait_all() waits for all of this thread's copies; a block
// barrier afterwards makes them visible to the other threads.
__device__ __forceinline__ void top_cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
// 8-byte variant (cached in L1 and L2); both addresses 8-byte aligned.
__device__ __forceinline__ void top_cp_async8(void* smem_dst, const void* gsrc) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void top_cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Close this thread's current group of copies; top_cp_async_wait_group<N>() waits until at most
// the N most recent groups are still in flight.
__device__ __forceinline__ void top_cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void top_cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
#endif

#ifndef TOP_L2_PREFETCH
#define TOP_L2_PREFETCH
// Bring `bytes` (a multiple of 16) from a 16-byte aligned global address into L2, asynchronously.
__device__ __forceinline__ void top_prefetch_l2(const void* gsrc, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gsrc), "r"(bytes) : "memory");
}
#endif

#ifndef TOP_NAMED_BARRIER
#define TOP_NAMED_BARRIER
// Barrier `id` (1..15) among `count` threads (a multiple of 32, whole warps) of the block.
__device__ __forceinline__ void top_named_barrier(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
#endif
