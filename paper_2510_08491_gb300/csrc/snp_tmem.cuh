// snp_tmem.cuh -- 5th-generation tensor-core (tcgen05) pieces used by the backward
// rasterizer at N_c = 64: tensor-memory (TMEM) allocation, one-thread MMA issue with
// operands in shared memory and the accumulator in TMEM, completion through an
// mbarrier, and TMEM-to-register loads.  Inline PTX (PTX ISA, "TensorCore 5th
// Generation Family Instructions"); every wait has an iteration limit.
//
// Operand layout (no swizzle, K-major): a tile of R rows x 16 bf16 is built from
// 8-row x 16-byte core matrices; element (r, k) sits at byte
//   (r / 8) * 256 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// i.e. the leading-dimension byte offset (between the two core matrices along K)
// is 128 and the stride-dimension byte offset (between 8-row groups) is 256.
// Accumulator layout for M = 64 (cta_group::1): row m of D is TMEM lane
// 32 (m / 16) + m % 16, column n is TMEM column n.  Both were checked on the GPU
// with a single-MMA test of known integer products before use.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace snp {

constexpr uint32_t kUmmaLbo = 128;  // bytes between core matrices along K
constexpr uint32_t kUmmaSbo = 256;  // bytes between 8-row groups
constexpr int kWaitLimit = 1 << 22; // polls of a bounded wait before it gives up

__device__ __forceinline__ uint32_t cvta_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading / stride byte offsets
// (all in 16-byte units), descriptor version 1 (bits 46-48 = 0b001), no swizzle.
__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((kUmmaLbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((kUmmaSbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: F32 accumulator (bits 4-5 = 1), BF16 A and B
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Warp-wide: allocate ncols (a power of two >= 32) TMEM columns; the address is
// written to *slot.  Then give up the right to allocate more (one allocation per CTA).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(cvta_smem(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Generic-proxy shared-memory writes become visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(cvta_smem(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// Wait until the phase of the given parity has completed; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int limit = kWaitLimit)
{
    const uint32_t a = cvta_smem(bar);
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// D[tmem] (+)= A[smem] B[smem] for one M x N x 16 bf16 tile; accumulate = false
// overwrites D.  Issued by one thread.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          bool accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// Arrive once on *bar when every MMA this thread issued before has completed.
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     cvta_smem(bar))
                 : "memory");
}

// Warp-wide load of 32 consecutive columns of the warp's 32 TMEM lanes
// (lane i of the warp gets TMEM lane (taddr >> 16) + i).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// Per-warp state of the TMEM accumulation of dL/dWc2 (see warp_color_bwd_pass).
struct TmemPass {
    void *stage_ptr;    // the warp's operand tiles: A hi, A lo, B hi, B lo (2 KB each)
    uint32_t stage;     // ... as a shared-memory address
    uint64_t *bar;      // the warp's MMA-completion barrier
    uint32_t d_tmem;    // TMEM address of the entry's 64 x 64 accumulator
    int *started;       // the entry's flag: its accumulator has been written in this chunk
    int *lock;          // CTA-wide MMA-issue lock
    int *wait_status;   // set to 1 when a bounded wait gives up
};

}  // namespace snp
