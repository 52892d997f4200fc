// Split-precision history sum, T_0 solve and projector apply on the 5th-generation tensor cores
// (tcgen05 + TMEM + TMA), sm_103a.
//
// Every matrix-times-block-of-vectors product of a step has the form
//     out[r][i] = sum_q sum_j A_q[i][j] x_q[r][j]            (r < R right-hand sides)
// with A_q = A_hi + A_lo and x = x_hi + x_lo split into 16-bit halves (x - hi rounded again).
// The three products A_hi x_hi + A_hi x_lo + A_lo x_hi are accumulated in FP32 in tensor memory;
// the lo*lo term is dropped.  Two formats:
//   BF16X3: bf16 halves, no scaling (about 2^-16 relative per stored entry);
//   FP16X3: fp16 halves of power-of-two scaled values (row scale per block for A, one scale per
//           slot and right-hand side for x; about 2^-22 relative per stored entry); the exact
//           inverse scales are applied in the epilogue.
//
// Kernel layout (one CTA per SM, persistent, 192 threads):
//   warp 0   TMA producer: A tiles (128 x 64, 128B swizzle) with L2 evict-first, x tiles
//            (R x 64) with L2 evict-last, into a STAGES-deep ring of shared-memory stages;
//   warp 1   one elected thread issues tcgen05.mma (M = 128, N = R, K = 16) and commits each
//            stage back to the producer and each finished accumulator to the epilogue;
//   warps 2-5 epilogue: after every chunk (at most CHUNK_KT k tiles of one block q), tcgen05.ld
//            of the 128 x R FP32 accumulator (two TMEM buffers, so the next chunk's MMAs
//            overlap), scaling by the block's row and slot scales, error-free accumulation in
//            registers (hi + lo pairs, TwoSum), and at a row-tile boundary a coalesced store of
//            the partial sum.  The MOT post-processing differences consecutive y, which magnifies
//            per-step errors of y about |y| / |y_n - y_{n-1}| times, so a long FP32 chain in
//            tensor memory would dominate the error at small time steps.
// Work split: stream-K over (row tile, q, k tile) iterations in row-tile-major order; a CTA's
// contiguous range covers parts of at most a few row tiles ("segments").  A second kernel sums
// the segment partials of every row tile in a fixed order (deterministic) and applies the
// step's epilogue.  Every mbarrier wait is bounded (%globaltimer, 2 s) and reports a timeout.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "plan.h"
#include "umma.h"

namespace tdc {

constexpr int BM = 128;      // rows per tile (UMMA M)
constexpr int BK = 64;       // bf16 elements per 128-byte row of a tile
constexpr int STAGES = 4;
constexpr int NTHREADS = 192;
constexpr uint64_t WAIT_NS = 2000000000ull;

template <int N>
struct Cfg {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = N * BK * 2;
    static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int SMEM = STAGES * STAGE + 1024 /*align*/ + 256 /*barriers*/;
    static constexpr int TMEM_COLS = 2 * N < 32 ? 32 : 2 * N;
};

struct GemmArgs {
    int rows, cols;       // M extent, K extent of one block
    int nblk, ktiles, rtiles;
    int64_t total;        // rtiles * nblk * ktiles
    int maxseg;
    int slot_mode;        // 0: history (q=0 -> slot ring, q=1 -> ring+1, q>=2 -> (n-(q-1)) mod ring); 1: slot 0
    int ring;
    float* partial;       // [grid][maxseg][N][BM]
    Ctl* ctl;
    uint32_t idesc;       // instruction descriptor (operand format)
    const float* sA;      // [nblk][rows] inverse row scales of A (nullptr: 1)
    const float* sX;      // [slots][N] inverse scales of x (nullptr: 1)
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false (and the step's timeout flag set) if the phase did not complete in WAIT_NS
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, Ctl* ctl) {
    if (mbar_try(b, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_try(b, parity)) {
        if (gtimer() - t0 > WAIT_NS) {
            atomicExch(&ctl->timeout, 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar,
                                            uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(const void* tile) {
    const uint64_t addr = smem_u32(tile);
    uint64_t d = 0;
    d |= (addr & 0x3FFFFull) >> 4;          // start address
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// instruction descriptor: kind::f16, (bf16 or fp16) x same -> f32, K-major A and B, M = 128, N
static uint32_t make_idesc(int n, bool bf16) {
    const uint32_t f = bf16 ? 1u : 0u;
    return (1u << 4) | (f << 7) | (f << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ int slot_of(const GemmArgs& g, int q, int64_t n) {
    if (g.slot_mode != 0) return 0;
    if (q == 0) return g.ring;
    if (q == 1) return g.ring + 1;
    int64_t sl = (n - (q - 1)) % g.ring;
    if (sl < 0) sl += g.ring;
    return (int)sl;
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 lanes x 32 columns of 32-bit values per warp (one lane = one row per thread)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Accumulator chunks: the MMA warp and the epilogue walk the same sequence of chunks, each at most
// CHUNK_KT k tiles of one (row tile, block q); a chunk never spans two blocks, so the block's row
// and slot scales apply to the whole chunk.  Short chunks keep the FP32 accumulation chain in
// tensor memory short; the epilogue sums the chunks error-free (hi + lo pairs and TwoSum).
constexpr int CHUNK_KT = 2;

__device__ __forceinline__ int64_t chunk_end(int64_t it, int64_t end, int ktiles) {
    const int64_t kt = it % ktiles;
    const int64_t qend = it - kt + ktiles;
    const int64_t cend = it - kt + (kt / CHUNK_KT + 1) * CHUNK_KT;
    const int64_t e = cend < qend ? cend : qend;
    return e < end ? e : end;
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
    const float t = hi + v;
    const float bp = t - hi;
    lo += (hi - (t - bp)) + (v - bp);
    hi = t;
}

// ---------------------------------------------------------------- the GEMM kernel
template <int N>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_umma_bf16x3(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                  const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl, GemmArgs g) {
    using C = Cfg<N>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * C::STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;     // [2]
    uint64_t* acc_empty = acc_full + 2;      // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int64_t ipt = (int64_t)g.nblk * g.ktiles;     // iterations per row tile
    const int64_t begin = (int64_t)blockIdx.x * g.total / gridDim.x;
    const int64_t end = (int64_t)(blockIdx.x + 1) * g.total / gridDim.x;
    Ctl* ctl = g.ctl;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(acc_full + b, 1); mbar_init(acc_empty + b, 128); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t n = ctl->n;

    if (warp == 0) {
        if (lane == 0) {
            const uint64_t pa = policy_evict_first(), pb = policy_evict_last();
            int stage = 0;
            uint32_t phase = 0;
            for (int64_t it = begin; it < end; ++it) {
                const int rt = (int)(it / ipt);
                const int64_t rem = it - rt * ipt;
                const int q = (int)(rem / g.ktiles), kt = (int)(rem - (int64_t)q * g.ktiles);
                const int slot = slot_of(g, q, n);
                if (!mbar_wait(empty + stage, phase ^ 1u, ctl)) break;
                uint8_t* st = smem + stage * C::STAGE;
                mbar_expect_tx(full + stage, C::STAGE);
                tma_load_3d(st, &tAh, kt * BK, rt * BM, q, full + stage, pa);
                tma_load_3d(st + C::A_BYTES, &tAl, kt * BK, rt * BM, q, full + stage, pa);
                tma_load_3d(st + 2 * C::A_BYTES, &tBh, kt * BK, 0, slot, full + stage, pb);
                tma_load_3d(st + 2 * C::A_BYTES + C::B_BYTES, &tBl, kt * BK, 0, slot, full + stage, pb);
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id = g.idesc;
            int stage = 0;
            uint32_t phase = 0;
            uint32_t ephase[2] = {0u, 0u};
            int chunk = 0;
            bool ok = true;
            // one accumulator per chunk (at most CHUNK_KT k tiles of one row tile and block q)
            for (int64_t it = begin; it < end && ok; ++chunk) {
                const int64_t cend = chunk_end(it, end, g.ktiles);
                const int buf = chunk & 1;
                if (!mbar_wait(acc_empty + buf, ephase[buf] ^ 1u, ctl)) { ok = false; break; }
                ephase[buf] ^= 1u;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * N);
                uint32_t acc = 0;
                for (; it < cend; ++it) {
                    if (!mbar_wait(full + stage, phase, ctl)) { ok = false; break; }
                    tc_fence_after();
                    uint8_t* st = smem + stage * C::STAGE;
                    const uint64_t ah = sdesc(st), al = sdesc(st + C::A_BYTES);
                    const uint64_t bh = sdesc(st + 2 * C::A_BYTES), bl = sdesc(st + 2 * C::A_BYTES + C::B_BYTES);
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k) {
                        const uint64_t adv = (uint64_t)(k * 32) >> 4;   // 16 elements = 32 bytes along K
                        umma(d, ah + adv, bh + adv, id, acc);
                        acc = 1;
                        umma(d, ah + adv, bl + adv, id, 1);
                        umma(d, al + adv, bh + adv, id, 1);
                    }
                    umma_commit(empty + stage);
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                umma_commit(acc_full + buf);
            }
        }
    } else {
        // epilogue warpgroup: warp w reads TMEM lanes 32 (w % 4) .. + 31 (one row per thread)
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        uint32_t fphase[2] = {0u, 0u};
        float acc_hi[N], acc_lo[N];
#pragma unroll
        for (int c = 0; c < N; ++c) acc_hi[c] = acc_lo[c] = 0.f;
        int chunk = 0, seg = 0;
        for (int64_t it = begin; it < end; ++chunk) {
            const int64_t cend = chunk_end(it, end, g.ktiles);
            const int64_t rt = it / ipt;
            const int q = (int)((it - rt * ipt) / g.ktiles);
            const int buf = chunk & 1;
            if (!mbar_wait(acc_full + buf, fphase[buf], ctl)) break;
            fphase[buf] ^= 1u;
            tc_fence_after();
            const int grow = (int)rt * BM + row;
            const float sa = (g.sA && grow < g.rows) ? g.sA[(int64_t)q * g.rows + grow] : 1.f;
            const float* sx = g.sX ? g.sX + (int64_t)slot_of(g, q, n) * N : nullptr;
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * N + c0), v);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 32; ++c)   // power-of-two scales: the products are exact
                    two_sum_acc(acc_hi[c0 + c], acc_lo[c0 + c], __uint_as_float(v[c]) * sa * (sx ? sx[c0 + c] : 1.f));
            }
            tc_fence_before();
            mbar_arrive(acc_empty + buf);
            it = cend;
            if (it == end || it % ipt == 0) {   // end of this CTA's part of row tile rt
                float* dst = g.partial + ((int64_t)blockIdx.x * g.maxseg + seg) * (int64_t)N * BM;
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    dst[(int64_t)c * BM + row] = acc_hi[c] + acc_lo[c];
                    acc_hi[c] = acc_lo[c] = 0.f;
                }
                ++seg;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------- partial-sum reduction + splits
// For row tile t, seg_ptr[t]..seg_ptr[t+1] lists the partial slots (cta * maxseg + seg) in a fixed
// order; out[r][row] (+ (n % 2) * R * rows when two_slots) receives their sum in FP32.
__global__ void k_fixup(const float* __restrict__ partial, const int* __restrict__ seg_ptr,
                        const int* __restrict__ seg_slot, int rows, int R, const Ctl* ctl, float* __restrict__ out,
                        int two_slots) {
    // grid (row tiles, R), BM threads: thread i sums the partials of row t*BM+i, right-hand side r
    const int t = blockIdx.x, r = blockIdx.y, i = threadIdx.x;
    const int row = t * BM + i;
    if (row >= rows) return;
    float* o = out + (two_slots ? (ctl->n % 2) * (int64_t)R * rows : 0);
    float s = 0.f;
    for (int k = seg_ptr[t]; k < seg_ptr[t + 1]; ++k) s += partial[(int64_t)seg_slot[k] * R * BM + (int64_t)r * BM + i];
    o[(int64_t)r * rows + row] = s;
}

__device__ __forceinline__ uint16_t to16(float v, bool fp16) {
    return fp16 ? __half_as_ushort(__float2half_rn(v)) : __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float from16(uint16_t b, bool fp16) {
    return fp16 ? __half2float(__ushort_as_half(b)) : __bfloat162float(__ushort_as_bfloat16(b));
}

// power of two p with m * p in (2^13, 2^14] (1 for m == 0): values scaled by p fill fp16 safely.
// The exponent is clamped to +-100 so that tiny vectors (e.g. an incident pulse that has passed,
// FP32 subnormals) cannot produce an infinite scale; such values then round to zero in fp16.
__device__ __forceinline__ float fill_scale(float m) {
    if (!(m > 0.f)) return 1.f;
    int e;
    frexpf(m, &e);             // m = f 2^e, f in [0.5, 1)
    int k = 14 - e;
    k = k > 100 ? 100 : (k < -100 ? -100 : k);
    return ldexpf(1.f, k);
}

// x: FP32 [R][n] (slot (n_step % 2) of a pair when pair != 0) -> 16-bit hi/lo [R][ld] into slot
// `slot` (slot < 0: n_step % ring) with one scale per right-hand side.  Grid (chunks, R): every
// block reduces the whole vector r to its maximum (cheap, from L2) and writes its chunk.
constexpr int SPLIT_CHUNK = 1024;
__global__ void k_split_vec(const float* __restrict__ x, int n, int R, int ld, uint16_t* __restrict__ hi,
                            uint16_t* __restrict__ lo, float* __restrict__ inv_scale, int slot, int ring, int pair,
                            int fp16, const Ctl* ctl) {
    __shared__ float red[256];
    const int r = blockIdx.y;
    const int64_t step = ctl->n;
    const float* xr = x + (pair ? (step % 2) * (int64_t)R * n : 0) + (int64_t)r * n;
    const int sl = slot >= 0 ? slot : (int)(step % ring);
    float sc = 1.f;
    if (fp16) {
        float m = 0.f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, fabsf(xr[i]));
        red[threadIdx.x] = m;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
            __syncthreads();
        }
        sc = fill_scale(red[0]);
    }
    const int64_t off = (int64_t)sl * R * ld + (int64_t)r * ld;
    const int i0 = blockIdx.x * SPLIT_CHUNK, i1 = min(n, i0 + SPLIT_CHUNK);
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const float v = xr[i] * sc;
        const uint16_t h = to16(v, fp16);
        hi[off + i] = h;
        lo[off + i] = to16(v - from16(h, fp16), fp16);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && inv_scale) inv_scale[(int64_t)sl * R + r] = 1.f / sc;
}

// FP64 matrix block (rows x cols, times `scale`) -> 16-bit hi/lo [rows][ld], zero padding;
// fp16: each row scaled by a power of two (inverse stored in inv_row).  One block per row.
__global__ void k_split_mat(const double* __restrict__ A, int rows, int cols, int ld, double scale,
                            uint16_t* __restrict__ hi, uint16_t* __restrict__ lo, float* __restrict__ inv_row,
                            int fp16) {
    __shared__ double red[256];
    const int r = blockIdx.x;
    const double* a = A + (int64_t)r * cols;
    double m = 0.0;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) m = fmax(m, fabs(scale * a[c]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    const float sc = fp16 ? fill_scale((float)red[0]) : 1.f;
    for (int c = threadIdx.x; c < ld; c += blockDim.x) {
        const double v = c < cols ? scale * a[c] * (double)sc : 0.0;
        const uint16_t h = to16((float)v, fp16);
        hi[(int64_t)r * ld + c] = h;
        lo[(int64_t)r * ld + c] = to16((float)(v - (double)from16(h, fp16)), fp16);
    }
    if (threadIdx.x == 0 && inv_row) inv_row[r] = 1.f / sc;
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
    }
    return fn;
}

// 3-D 16-bit map {inner (K), rows, slices} with box {64, box_rows, 1}, 128-byte swizzle
static bool make_map(CUtensorMap* m, void* base, int64_t inner, int64_t rows, int64_t slices, int64_t ld,
                     int box_rows, bool fp16) {
    EncodeTiled enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)slices};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * 2 * rows};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides,
               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct Gemm {
    CUtensorMap ah, al, bh, bl;
    GemmArgs a;
    int grid = 0;
    int* seg_ptr = nullptr;
    int* seg_slot = nullptr;
};

struct Bf16x3Gemm {
    bool fp16 = false;
    int ld = 0, ldc = 0, R = 0, sms = 0;
    uint16_t *Ah = nullptr, *Al = nullptr;          // history blocks [nblk][ne][ld]
    uint16_t *Th = nullptr, *Tl = nullptr;          // T_0^-1
    uint16_t *Ph = nullptr, *Pl = nullptr;          // (Sigma^T Sigma)^+
    uint16_t *Xh = nullptr, *Xl = nullptr;          // history ring + e_n + h_n slots [ring+2][R][ld]
    uint16_t *bh = nullptr, *bl = nullptr;          // b [R][ld]
    uint16_t *zh = nullptr, *zl = nullptr;          // z [R][ldc]
    float *sAh = nullptr, *sAs = nullptr, *sAp = nullptr;   // inverse row scales (fp16)
    float *sXh = nullptr, *sXb = nullptr, *sXz = nullptr;   // inverse vector scales (fp16)
    float *E = nullptr, *H = nullptr, *b32 = nullptr, *y32 = nullptr, *z32 = nullptr, *u32 = nullptr;
    float* partial = nullptr;
    Gemm hist, solve, proj;
    std::vector<void*> owned;
    ~Bf16x3Gemm() {
        for (void* p : owned) cudaFree(p);
        for (Gemm* g : {&hist, &solve, &proj}) {
            if (g->seg_ptr) cudaFree(g->seg_ptr);
            if (g->seg_slot) cudaFree(g->seg_slot);
        }
    }
};

void destroy_bf16x3(Bf16x3Gemm* g) { delete g; }

// history ring, e/h slots and the FP32 y pair start at zero (y_i = 0 for i <= 0)
cudaError_t reset_bf16x3(Bf16x3Gemm* g, int ring, cudaStream_t s) {
    const size_t xs = sizeof(uint16_t) * (size_t)(ring + 2) * g->R * g->ld;
    cudaError_t e;
    if ((e = cudaMemsetAsync(g->Xh, 0, xs, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(g->Xl, 0, xs, s)) != cudaSuccess) return e;
    return cudaMemsetAsync(g->y32, 0, sizeof(float) * 2 * (size_t)g->R * g->ld, s);
}

template <class T>
static cudaError_t dalloc(Bf16x3Gemm* g, T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) g->owned.push_back(*p);
    return e;
}

// stream-K partition and the per-row-tile list of partial slots (same traversal as the kernel)
static cudaError_t plan_gemm(Gemm& G, int rows, int cols, int nblk, int sms) {
    GemmArgs& a = G.a;
    a.rows = rows;
    a.cols = cols;
    a.nblk = nblk;
    a.ktiles = (cols + BK - 1) / BK;
    a.rtiles = (rows + BM - 1) / BM;
    a.total = (int64_t)a.rtiles * nblk * a.ktiles;
    G.grid = (int)std::min<int64_t>(sms, a.total);
    const int64_t ipt = (int64_t)nblk * a.ktiles;
    std::vector<std::vector<std::pair<int, int>>> lists(a.rtiles);
    int maxseg = 1;
    for (int c = 0; c < G.grid; ++c) {
        const int64_t b = (int64_t)c * a.total / G.grid, e = (int64_t)(c + 1) * a.total / G.grid;
        int seg = 0;
        for (int64_t it = b; it < e; ++seg) {
            const int64_t rt = it / ipt;
            lists[rt].push_back({c, seg});
            it = std::min<int64_t>(e, (rt + 1) * ipt);
        }
        maxseg = std::max(maxseg, seg);
    }
    a.maxseg = maxseg;
    std::vector<int> ptr(a.rtiles + 1, 0), slot;
    for (int t = 0; t < a.rtiles; ++t) {
        for (auto& cs : lists[t]) slot.push_back(cs.first * maxseg + cs.second);
        ptr[t + 1] = (int)slot.size();
    }
    cudaError_t e;
    if ((e = cudaMalloc(&G.seg_ptr, sizeof(int) * ptr.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc(&G.seg_slot, sizeof(int) * slot.size())) != cudaSuccess) return e;
    if ((e = cudaMemcpy(G.seg_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    return cudaMemcpy(G.seg_slot, slot.data(), sizeof(int) * slot.size(), cudaMemcpyHostToDevice);
}

#define CKB(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return cuda_fail(h, e_, #x); } while (0)

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

tdcfie_status build_bf16x3(tdcfie_t h, StepPlan* p) {
    const int R = p->R, ne = p->ne, nc = p->nc, K = h->K;
    if (R != 64) return fail(h, TDCFIE_E_UNSUPPORTED, "tensor-core path is built for R = 64 right-hand sides");
    if (!encoder()) return fail(h, TDCFIE_E_CUDA, "cuTensorMapEncodeTiled entry point not available");
    auto* g = new Bf16x3Gemm();
    p->gemm = g;
    g->fp16 = (p->prec == TDCFIE_FP16X3);
    const int f16 = g->fp16 ? 1 : 0;
    cudaStream_t s = h->stream;
    int dev = 0;
    CKB(cudaGetDevice(&dev));
    CKB(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev));
    g->R = R;
    g->ld = round_up(ne, BK);
    g->ldc = round_up(nc, BK);
    const int ld = g->ld, ldc = g->ldc, nblk = p->nblk, ring = p->ring;
    const size_t blk = (size_t)ne * ld;
    CKB(dalloc(g, &g->Ah, blk * nblk));
    CKB(dalloc(g, &g->Al, blk * nblk));
    CKB(dalloc(g, &g->Th, blk));
    CKB(dalloc(g, &g->Tl, blk));
    CKB(dalloc(g, &g->Ph, (size_t)nc * ldc));
    CKB(dalloc(g, &g->Pl, (size_t)nc * ldc));
    CKB(dalloc(g, &g->Xh, (size_t)(ring + 2) * R * ld));
    CKB(dalloc(g, &g->Xl, (size_t)(ring + 2) * R * ld));
    CKB(dalloc(g, &g->bh, (size_t)R * ld));
    CKB(dalloc(g, &g->bl, (size_t)R * ld));
    CKB(dalloc(g, &g->zh, (size_t)R * ldc));
    CKB(dalloc(g, &g->zl, (size_t)R * ldc));
    CKB(dalloc(g, &g->E, (size_t)R * ne));
    CKB(dalloc(g, &g->H, (size_t)R * ne));
    CKB(dalloc(g, &g->b32, (size_t)R * ne));
    CKB(dalloc(g, &g->y32, (size_t)2 * R * ld));
    CKB(dalloc(g, &g->z32, (size_t)R * nc));
    CKB(dalloc(g, &g->u32, (size_t)R * nc));
    if (g->fp16) {
        CKB(dalloc(g, &g->sAh, (size_t)nblk * ne));
        CKB(dalloc(g, &g->sAs, (size_t)ne));
        CKB(dalloc(g, &g->sAp, (size_t)nc));
        CKB(dalloc(g, &g->sXh, (size_t)(ring + 2) * R));
        CKB(dalloc(g, &g->sXb, (size_t)R));
        CKB(dalloc(g, &g->sXz, (size_t)R));
        std::vector<float> ones((size_t)(ring + 2) * R, 1.f);
        CKB(cudaMemcpy(g->sXh, ones.data(), sizeof(float) * ones.size(), cudaMemcpyHostToDevice));
    }
    for (void* q : {(void*)g->Xh, (void*)g->Xl}) CKB(cudaMemsetAsync(q, 0, sizeof(uint16_t) * (ring + 2) * R * ld, s));
    for (void* q : {(void*)g->bh, (void*)g->bl}) CKB(cudaMemsetAsync(q, 0, sizeof(uint16_t) * R * ld, s));
    for (void* q : {(void*)g->zh, (void*)g->zl}) CKB(cudaMemsetAsync(q, 0, sizeof(uint16_t) * R * ldc, s));
    // matrices: -A, alpha L2, -T_1 .. -T_{K-1}, then T_0^-1 and the Laplacian pseudo-inverse
    const int64_t NN = (int64_t)ne * ne;
    auto rows_scale = [&](float* base, int q) { return base ? base + (int64_t)q * ne : nullptr; };
    k_split_mat<<<ne, 256, 0, s>>>(h->A, ne, ne, ld, -1.0, g->Ah, g->Al, rows_scale(g->sAh, 0), f16);
    k_split_mat<<<ne, 256, 0, s>>>(h->L2, ne, ne, ld, h->alpha, g->Ah + blk, g->Al + blk, rows_scale(g->sAh, 1), f16);
    for (int k = 1; k < K; ++k)
        k_split_mat<<<ne, 256, 0, s>>>(h->T + k * NN, ne, ne, ld, -1.0, g->Ah + (1 + k) * blk, g->Al + (1 + k) * blk,
                                       rows_scale(g->sAh, 1 + k), f16);
    k_split_mat<<<ne, 256, 0, s>>>(h->T0inv, ne, ne, ld, 1.0, g->Th, g->Tl, g->sAs, f16);
    k_split_mat<<<nc, 256, 0, s>>>(h->PinvS, nc, nc, ldc, 1.0, g->Ph, g->Pl, g->sAp, f16);
    CKB(cudaGetLastError());
    // GEMM plans and tensor maps
    CKB(plan_gemm(g->hist, ne, ne, nblk, g->sms));
    CKB(plan_gemm(g->solve, ne, ne, 1, g->sms));
    CKB(plan_gemm(g->proj, nc, nc, 1, g->sms));
    size_t pmax = 0;
    for (Gemm* G : {&g->hist, &g->solve, &g->proj}) pmax = std::max(pmax, (size_t)G->grid * G->a.maxseg * BM * R);
    CKB(dalloc(g, &g->partial, pmax));
    const bool fp = g->fp16;
    bool ok = make_map(&g->hist.ah, g->Ah, ne, ne, nblk, ld, BM, fp) && make_map(&g->hist.al, g->Al, ne, ne, nblk, ld, BM, fp) &&
              make_map(&g->hist.bh, g->Xh, ne, R, ring + 2, ld, R, fp) &&
              make_map(&g->hist.bl, g->Xl, ne, R, ring + 2, ld, R, fp) &&
              make_map(&g->solve.ah, g->Th, ne, ne, 1, ld, BM, fp) && make_map(&g->solve.al, g->Tl, ne, ne, 1, ld, BM, fp) &&
              make_map(&g->solve.bh, g->bh, ne, R, 1, ld, R, fp) && make_map(&g->solve.bl, g->bl, ne, R, 1, ld, R, fp) &&
              make_map(&g->proj.ah, g->Ph, nc, nc, 1, ldc, BM, fp) && make_map(&g->proj.al, g->Pl, nc, nc, 1, ldc, BM, fp) &&
              make_map(&g->proj.bh, g->zh, nc, R, 1, ldc, R, fp) && make_map(&g->proj.bl, g->zl, nc, R, 1, ldc, R, fp);
    if (!ok) return fail(h, TDCFIE_E_CUDA, "cuTensorMapEncodeTiled failed");
    const uint32_t id = make_idesc(R, !fp);
    for (Gemm* G : {&g->hist, &g->solve, &g->proj}) {
        G->a.partial = g->partial;
        G->a.ctl = p->ctl;
        G->a.ring = ring;
        G->a.slot_mode = 1;
        G->a.idesc = id;
    }
    g->hist.a.slot_mode = 0;
    g->hist.a.sA = g->sAh; g->hist.a.sX = g->sXh;
    g->solve.a.sA = g->sAs; g->solve.a.sX = g->sXb;
    g->proj.a.sA = g->sAp; g->proj.a.sX = g->sXz;
    CKB(cudaFuncSetAttribute(k_umma_bf16x3<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<64>::SMEM));
    CKB(cudaStreamSynchronize(s));
    // algorithmic bytes of the history GEMM: every block (hi + lo) once, and its R vectors
    h->hist_bytes = (double)nblk * ne * ne * 4.0 + (double)nblk * R * ne * 4.0;
    return TDCFIE_OK;
}

static void run_gemm(const Gemm& G, cudaStream_t s) {
    k_umma_bf16x3<64><<<G.grid, NTHREADS, Cfg<64>::SMEM, s>>>(G.ah, G.al, G.bh, G.bl, G.a);
}

void launch_step_bf16x3(tdcfie_t h, StepPlan* p, cudaStream_t s) {
    Bf16x3Gemm* g = p->gemm;
    const int R = p->R, ne = p->ne, nc = p->nc, ring = p->ring, ld = g->ld, ldc = g->ldc;
    const int f16 = g->fp16 ? 1 : 0;
    // plane-wave tests -> e, h slots of the history operand
    const dim3 gv((ne + SPLIT_CHUNK - 1) / SPLIT_CHUNK, R), gz((nc + SPLIT_CHUNK - 1) / SPLIT_CHUNK, R);
    launch_rhs_f32(h, p, g->E, g->H, s);
    k_split_vec<<<gv, 256, 0, s>>>(g->E, ne, R, ld, g->Xh, g->Xl, g->sXh, ring, ring, 0, f16, p->ctl);
    k_split_vec<<<gv, 256, 0, s>>>(g->H, ne, R, ld, g->Xh, g->Xl, g->sXh, ring + 1, ring, 0, f16, p->ctl);
    // history sum b_n = -A e_n + alpha L2 h_n - sum_k T_k y_{n-k}  (events bracket the GEMM alone)
    cudaEventRecordWithFlags(p->evA, s, cudaEventRecordExternal);
    run_gemm(g->hist, s);
    cudaEventRecordWithFlags(p->evB, s, cudaEventRecordExternal);
    k_fixup<<<dim3(g->hist.a.rtiles, R), BM, 0, s>>>(g->partial, g->hist.seg_ptr, g->hist.seg_slot, ne, R, p->ctl,
                                                     g->b32, 0);
    k_split_vec<<<gv, 256, 0, s>>>(g->b32, ne, R, ld, g->bh, g->bl, g->sXb, 0, ring, 0, f16, p->ctl);
    // y_n = T_0^-1 b_n  (FP32 in y32[n % 2]; 16-bit hi/lo into history slot n % ring)
    run_gemm(g->solve, s);
    k_fixup<<<dim3(g->solve.a.rtiles, R), BM, 0, s>>>(g->partial, g->solve.seg_ptr, g->solve.seg_slot, ne, R,
                                                      p->ctl, g->y32, 1);
    k_split_vec<<<gv, 256, 0, s>>>(g->y32, ne, R, ld, g->Xh, g->Xl, g->sXh, -1, ring, 1, f16, p->ctl);
    // projector: z = Sigma^T w_n, u = (Sigma^T Sigma)^+ z, j_n = y_n + Sigma u
    launch_project_in_f32(h, p, g->y32, 2, g->z32, s);
    k_split_vec<<<gz, 256, 0, s>>>(g->z32, nc, R, ldc, g->zh, g->zl, g->sXz, 0, ring, 0, f16, p->ctl);
    run_gemm(g->proj, s);
    k_fixup<<<dim3(g->proj.a.rtiles, R), BM, 0, s>>>(g->partial, g->proj.seg_ptr, g->proj.seg_slot, nc, R, p->ctl,
                                                     g->u32, 0);
    launch_project_out_f32(h, p, g->y32, 2, g->u32, s);
    launch_advance(p, s);
    p->launches_per_step = 16;
}

}  // namespace tdc
