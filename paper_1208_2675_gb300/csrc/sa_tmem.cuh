// sa_tmem.cuh -- Tensor Memory (TMEM) as the home of a CTA's Delta cells.
//
// Each SM of sm_100/sm_103 has 256 KB of TMEM: 128 lanes x 512 columns of 32-bit
// cells, allocated per CTA in power-of-two column counts and accessed with
// warp-collective tcgen05.ld / tcgen05.st.  Warp w of a CTA reaches the 32 lanes
// 32*(w % 4) .. 32*(w % 4) + 31; in the 32x32b shape lane k of that range is
// thread k of the warp, and an .xN access moves N consecutive columns of it into
// N registers of that thread.  The SA kernels keep each thread's R x 4 tile of
// Delta in its own lane, in 4R consecutive columns, so that the tiles no longer
// occupy registers (where, with 640 threads and 96 registers a thread, they
// forced spills) and are moved in and out in 16- or 32-column pieces.
//
// Every load is waited for inside the same asm statement, so the compiler never
// sees a register of an unfinished load; every store likewise, so a later load
// of the same columns by the same thread sees it.  The tcgen05 instructions are
// warp-collective (.sync.aligned) and the compiler does not know that of an asm
// statement, so each helper first reconverges the warp with __syncwarp(); every
// caller reaches them with all 32 threads.
#pragma once
#include <cstdint>

namespace qapsa {

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Allocates ncols columns (a power of two, 32..512) for the calling CTA; the
// whole warp must call it.  The TMEM address is written to *dst (shared).
__device__ __forceinline__ void tmem_alloc(unsigned *dst, unsigned ncols) {
  __syncwarp();
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               :: "r"(smem_u32(dst)), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Frees what tmem_alloc gave; the whole warp must call it.
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
  __syncwarp();
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
               :: "r"(taddr), "r"(ncols) : "memory");
}

// Orders TMEM accesses before / after a thread barrier.
__device__ __forceinline__ void tmem_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// TMEM address of the calling warp's lanes at column col (base from tmem_alloc).
__device__ __forceinline__ unsigned tmem_warp_addr(unsigned base, int warp, int col) {
  return base + ((unsigned)((warp & 3) * 32) << 16) + (unsigned)col;
}

// 16 consecutive columns of this thread's lane -> v[0..15] (warp-collective).
__device__ __forceinline__ void tmem_ld16(unsigned taddr, int (&v)[16]) {
  __syncwarp();
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
        "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
        "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

// v[0..15] -> 16 consecutive columns of this thread's lane (warp-collective).
__device__ __forceinline__ void tmem_st16(unsigned taddr, const int (&v)[16]) {
  __syncwarp();
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};\n\t"
      "tcgen05.wait::st.sync.aligned;"
      :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
         "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]),
         "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

// 32 consecutive columns of this thread's lane -> v[0..31] (warp-collective).
__device__ __forceinline__ void tmem_ld32(unsigned taddr, int (&v)[32]) {
  __syncwarp();
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
      "[%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
        "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
        "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
        "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
        "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}

// v[0..31] -> 32 consecutive columns of this thread's lane (warp-collective).
__device__ __forceinline__ void tmem_st32(unsigned taddr, const int (&v)[32]) {
  __syncwarp();
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n\t"
      "tcgen05.wait::st.sync.aligned;"
      :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
         "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]),
         "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
         "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
         "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]),
         "r"(v[31])
      : "memory");
}

// Columns a CTA of the SA kernels allocates: all 512.  With 64 columns a thread
// (one 16 x 4 tile) and warps w, w+4, w+8, ... sharing a lane group, a block of
// up to 1024 threads fits.  Only one such CTA is resident on an SM: they all run
// 640 threads at more than 51 registers each, or (the cluster kernels) use more
// than half of the SM's shared memory; a second CTA that asked for TMEM would
// wait in tcgen05.alloc until the first one freed it.
constexpr unsigned kTileTmemCols = 512;

// TMEM for the calling CTA's tiles: allocated by warp 0, the address passed
// through shared memory; returns the address of this thread's tile
// (cols_per_thread consecutive columns of its lane).
__device__ __forceinline__ unsigned tile_tmem_acquire(unsigned *s_tmem, int cols_per_thread) {
  if (threadIdx.x < 32) tmem_alloc(s_tmem, kTileTmemCols);
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const int warp = (int)(threadIdx.x >> 5);
  return tmem_warp_addr(*s_tmem, warp, (warp >> 2) * cols_per_thread);
}

// Every TMEM access of the CTA is done; warp 0 frees the columns.
__device__ __forceinline__ void tile_tmem_release(const unsigned *s_tmem) {
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (threadIdx.x < 32) tmem_dealloc(*s_tmem, kTileTmemCols);
}

}  // namespace qapsa
