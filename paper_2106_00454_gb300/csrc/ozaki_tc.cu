// ozaki_tc.cu -- the digit-pair products of the Ozaki scheme (ozaki.cu) on the
// fifth-generation tensor cores: TMA loads, tcgen05.mma, accumulators in tensor
// memory (TMEM).
//
// A persistent kernel, one CTA per SM, walks the 128 x 64 output tiles of
// C[b] = A[b] B[b] (A: row slices, B: column slices, both k-contiguous).  Its
// eighteen warps split the work:
//   * warp 16 (one thread) streams k-chunks of 32 through a 3-stage ring: one
//     TMA box per operand brings all six digits of the chunk (128 rows of A,
//     64 columns of B; 72 KB), in the 64-byte-swizzled K-major layout the
//     tensor core reads;
//   * warp 17 (one thread) owns the tensor memory and issues, per 16-k step,
//     the 21 digit pairs p + q <= 5 into six FP32 accumulators, one per weight
//     d = p + q (6 x 64 TMEM columns), as eight M = 128, K = 16 MMAs of
//     N = 64 .. 256 that each multiply one A digit by up to four adjacent B
//     digits.  A narrow last column tile takes the same eight MMAs over B rows
//     that the TMA zero-filled past n: a chain of small-N MMAs into one
//     accumulator is bound by the MMA latency and costs several times more
//     than the padded columns;
//   * warps 0-15 drain the accumulators every 160 k into per-thread int64
//     sums, shifted by 36 - 8d (warp w reads TMEM lanes 32 (w % 4) .. + 31 =
//     rows of the tile, columns 16 (w / 4) .. + 15), and write the FP64 tile
//     while the MMAs of the next k-block or tile proceed: each integer becomes
//     an IEEE-754 pattern with integer operations (exponent added afterwards,
//     so the 16 conversions of a thread are independent), and a butterfly of
//     warp shuffles turns the warp's rows into 128-byte row segments for
//     coalesced stores.  The drain (6 x 64 x 128 FP32 -> int conversions per
//     160 k and tile) is the part the MMAs wait for: the six accumulators take
//     384 of the 512 TMEM columns, too many to double; the warps hand the tensor
//     memory back as soon as the last pair of accumulators is in registers.
// Exactness: digit 0 lies in [-129, 129] and digits 1-5 in [-128, 127], so a
// weight-d accumulator (at most six digit pairs, two of them with digit 0)
// gains at most 2 * 129 * 128 + 4 * 128^2 = 99,560 per k; over 160 k that is
// 15,929,600 < 2^24, so every FP32 accumulator is an exact integer.  The int64
// sums stay below 2^61 for n <= 1024.
//
// Every mbarrier wait is bounded (about a second at the SM clock); on a timeout
// the kernel records kDevTimeout, the other roles stop at their next wait, the
// loads and MMAs in flight are waited for (bounded) and the tensor memory is
// freed before the CTA returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "wpcd_internal.cuh"

namespace wpcd {

// The IEEE-754 pattern of the int64 v as a double, rounded to 53 bits (half
// away from zero), from integer operations only and with no branch; 0 for
// v = 0.  Its exponent field lies in [1023, 1087]; a caller scaling by 2^e adds
// e << 52, which keeps the pattern normal for e in [-1022, 959].
__device__ __forceinline__ unsigned long long i64_to_f64_bits(long long v)
{
    const unsigned long long m = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)m);  // 64 for m = 0
    const unsigned long long mn = m << (lz & 63);
    const unsigned long long r = mn + 0x400ull;
    const bool carry = r < mn;  // the rounding carried out of the top bit
    const unsigned long long frac = carry ? 0ull : ((r >> 11) & ((1ull << 52) - 1));
    const unsigned long long be = (unsigned long long)(1086 - lz + (carry ? 1 : 0));  // 63 - lz + 1023
    const unsigned long long bits = (v < 0 ? (1ull << 63) : 0ull) | (be << 52) | frac;
    return m == 0 ? 0ull : bits;
}

// x 2^e for the rare tiles whose scale leaves the range above (out of line).
__device__ __noinline__ double f64_times_pow2_slow(double x, int e) { return ldexp(x, e); }

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

constexpr int kTcM = 128;       // tile rows = TMEM lanes
constexpr int kTcN = 64;        // tile columns = TMEM columns per accumulator
constexpr int kTcKC = 32;       // k per stage: 64 bytes of a row = one swizzle span
constexpr int kTcKBlk = 160;    // k between drains (exact FP32 sums)
constexpr int kTcStages = 3;
constexpr int kTcADigit = kTcM * kTcKC * 2;                        // 8 KB
constexpr int kTcBDigit = kTcN * kTcKC * 2;                        // 4 KB
constexpr int kTcAStage = kOzDigits * kTcADigit;                   // 48 KB
constexpr int kTcStageBytes = kOzDigits * (kTcADigit + kTcBDigit);  // 72 KB
constexpr int kTcTmemCols = 512;  // 6 x 64 accumulator columns, allocated as a power of two
constexpr int kTcDrainWarps = 16;  // four per TMEM lane quarter, one per 16 columns
constexpr int kTcDrainCols = kTcN / (kTcDrainWarps / 4);
constexpr int kTcProducerWarp = kTcDrainWarps, kTcMmaWarp = kTcDrainWarps + 1;
constexpr int kTcThreads = 32 * (kTcDrainWarps + 2);
constexpr int kTcSmem = 1024 + kTcStages * kTcStageBytes + 128;  // alignment slack | ring | barriers
constexpr long long kTcWaitCycles = 1ll << 31;

// instruction descriptor: D F32, A and B BF16, both K-major, M = 128; N (bits
// 17-22, N / 8) is set per MMA: 64 times the number of B digits it takes
constexpr uint32_t kTcIdescBase = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcM >> 4) << 24);

// The 21 digit pairs of one 16-k step as eight wide MMAs.  The B digits of a
// stage lie back to back in shared memory (64 rows each, the same 512-byte
// row-group stride), so digits q0 .. q0 + nq - 1 form one K-major operand of
// N = 64 nq rows; A digit p times it lands, 64 columns per digit, on the
// accumulators of weights p + q0 .. p + q0 + nq - 1, which are adjacent in
// TMEM.  Segment g = (p, q0, nq): every pair p + q <= 5 exactly once, and the
// two p = 0 segments write every weight before any other segment does.
constexpr int kTcSegs = 8;
__device__ __forceinline__ void tc_seg(int g, int &p, int &q0, int &nq)
{
    constexpr int P[kTcSegs] = {0, 0, 1, 1, 2, 3, 4, 5};
    constexpr int Q0[kTcSegs] = {0, 4, 0, 4, 0, 0, 0, 0};
    constexpr int NQ[kTcSegs] = {4, 2, 4, 1, 4, 3, 2, 1};
    p = P[g];
    q0 = Q0[g];
    nq = NQ[g];
}

__device__ __forceinline__ int tc_tile_n(int n, int col0)
{
    const int w = (n - col0 + 15) & ~15;
    return w < kTcN ? w : kTcN;
}

// Shared-memory matrix descriptor of a K-major operand with 64-byte swizzle:
// rows of 64 bytes, 8-row groups 512 bytes apart (stride offset); the leading
// offset is unused when one MMA's K (32 bytes) stays inside the swizzle span.
__device__ __forceinline__ uint64_t tc_desc_sw64(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused): 16 B
    d |= (uint64_t)(512 >> 4) << 32;      // stride byte offset: 512 B
    d |= (uint64_t)1 << 46;               // descriptor version of this architecture
    d |= (uint64_t)4 << 61;               // layout: 64-byte swizzle
    return d;
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the completion of the phase with the given parity; gives up
// early when another role has aborted (abort != nullptr).
__device__ __forceinline__ bool tc_wait(uint32_t a, uint32_t parity, const volatile int *abort)
{
    if (mbar_try(a, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(a, parity)) {
        if (abort && *abort) return false;
        if (clock64() - t0 > kTcWaitCycles) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint32_t a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Transpose the 16 x 16 blocks held one row per lane in each half-warp
// (v[j] = M[lane % 16][j]) into one column per lane (v[j] = M[j][lane % 16]):
// four butterfly stages, each swapping the off-diagonal s x s sub-blocks of
// every 2s x 2s block between lanes l and l ^ s.
__device__ __forceinline__ void tc_transpose16(double (&v)[16], int lane)
{
#pragma unroll
    for (int s = 8; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j & s) continue;
            const double send = up ? v[j] : v[j + s];
            const double recv = __shfl_xor_sync(0xffffffffu, send, s);
            if (up) v[j] = recv;
            else v[j + s] = recv;
        }
    }
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct TcTile {
    int b, row0, col0;
};

// Tile t of the launch: item-major; per item the row tiles (128) x column tiles
// (64), or for a symmetric product only those reaching the diagonal or above it
// (column tiles 2 tr .. TC - 1 of row tile tr).
__device__ __forceinline__ TcTile tc_tile(int t, int per_item, int TC, bool sym)
{
    TcTile r;
    r.b = t / per_item;
    int j = t - r.b * per_item;
    int tr = 0;
    if (sym) {
        while (j >= TC - 2 * tr) {
            j -= TC - 2 * tr;
            ++tr;
        }
        j += 2 * tr;
    } else {
        tr = j / TC;
        j -= tr * TC;
    }
    r.row0 = tr * kTcM;
    r.col0 = j * kTcN;
    return r;
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_oz_gemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int n, int Kp,
                 int dmax, bool sym, int per_item, int TC, int ntiles, const int *ea_all, const int *eb_all,
                 double *C_all, int *err, int a_mod)
{
    extern __shared__ unsigned char tc_raw[];
    const uint32_t raw_s = smem_u32(tc_raw);
    const uint32_t ring_s = (raw_s + 1023u) & ~1023u;  // the swizzle pattern follows address bits
    unsigned char *ring = tc_raw + (ring_s - raw_s);
    const uint32_t bar_s = ring_s + kTcStages * kTcStageBytes;
    // barriers: full[3] | empty[3] | acc_full | acc_empty, then the TMEM base and the abort flag
    const uint32_t full_s = bar_s, empty_s = bar_s + 8u * kTcStages;
    const uint32_t accf_s = bar_s + 16u * kTcStages, acce_s = accf_s + 8u;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(ring + kTcStages * kTcStageBytes + 64);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < 2 * kTcStages + 1; ++i) mbar_init(bar_s + 8u * i, 1);
        mbar_init(acce_s, 32 * kTcDrainWarps);  // every drain thread arrives
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kTcMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool failed = false;

    if (warp == kTcProducerWarp) {
        // ---- producer: TMA of every k-chunk of every tile of this CTA
        if (lane == 0) {
            int stage = 0, issued = 0;
            uint32_t ph = 0;
            for (int t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
                const TcTile tl = tc_tile(t, per_item, TC, sym);
                for (int k0 = 0; k0 < Kp; k0 += kTcKC) {
                    if (!tc_wait(empty_s + 8u * stage, ph ^ 1u, abort_flag)) {
                        failed = true;
                        break;
                    }
                    const uint32_t sA = ring_s + (uint32_t)(stage * kTcStageBytes);
                    mbar_expect_tx(full_s + 8u * stage, (uint32_t)kTcStageBytes);
                    tma_load_3d(sA, &mapA, k0, tl.row0, (tl.b % a_mod) * kOzDigits, full_s + 8u * stage);
                    tma_load_3d(sA + kTcAStage, &mapB, k0, tl.col0, tl.b * kOzDigits, full_s + 8u * stage);
                    ++issued;
                    if (++stage == kTcStages) {
                        stage = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (failed) {
                *abort_flag = 1;
                // the copies still in flight land before the shared memory is released
                for (int i = issued - 1; i >= 0 && i >= issued - kTcStages; --i)
                    tc_wait(full_s + 8u * (i % kTcStages), (uint32_t)((i / kTcStages) & 1), nullptr);
            }
        }
    } else if (warp == kTcMmaWarp) {
        // ---- MMA issuer
        if (lane == 0) {
            int stage = 0, blk = 0, committed = 0;
            uint32_t ph = 0;
            for (int t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
                const TcTile tl = tc_tile(t, per_item, TC, sym);
                for (int k0 = 0; k0 < Kp; k0 += kTcKC) {
                    const bool bfirst = (k0 % kTcKBlk) == 0;
                    const bool blast = ((k0 + kTcKC) % kTcKBlk) == 0 || k0 + kTcKC >= Kp;
                    if (bfirst && blk > 0 && !tc_wait(acce_s, (uint32_t)((blk - 1) & 1), abort_flag)) {
                        failed = true;  // the accumulators were not drained
                        break;
                    }
                    if (!tc_wait(full_s + 8u * stage, ph, abort_flag)) {
                        failed = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sA = ring_s + (uint32_t)(stage * kTcStageBytes), sB = sA + kTcAStage;
                    const uint64_t a0 = tc_desc_sw64(sA), b0 = tc_desc_sw64(sB);
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {  // K = 16: 32 bytes further into the swizzle span
                        if (kk == 1 && k0 + 16 >= n) break;  // that half of the chunk is zero padding
#pragma unroll
                        for (int g = 0; g < kTcSegs; ++g) {
                            int p, q0, nq;
                            tc_seg(g, p, q0, nq);
                            nq = min(nq, dmax - p - q0 + 1);
                            if (nq <= 0) continue;
                            const uint64_t ad = a0 + (uint64_t)((p * kTcADigit + kk * 32) >> 4);
                            const uint64_t bd = b0 + (uint64_t)((q0 * kTcBDigit + kk * 32) >> 4);
                            tc_mma(tmem + (uint32_t)((p + q0) * kTcN), ad, bd,
                                   kTcIdescBase | ((uint32_t)(nq * kTcN >> 3) << 17),
                                   (bfirst && kk == 0 && p == 0) ? 0u : 1u);
                        }
                    }
                    tc_commit(empty_s + 8u * stage);
                    ++committed;
                    if (blast) {
                        tc_commit(accf_s);
                        ++blk;
                    }
                    if (++stage == kTcStages) {
                        stage = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (failed) {
                *abort_flag = 1;
                // commits complete in order: the last one covers every MMA issued
                if (committed > 0)
                    tc_wait(empty_s + 8u * ((committed - 1) % kTcStages),
                            (uint32_t)(((committed - 1) / kTcStages) & 1), nullptr);
            }
        }
        __syncwarp();
    } else {
        // ---- drain and epilogue: rows rbase .. + 31 of the tile (TMEM lane quarter
        // warp % 4, one row per lane), columns c0 .. c0 + 15
        static_assert(kTcDrainCols == 16, "the drain and its transpose take 16 columns per warp");
        int blk = 0;
        const int c0 = (warp >> 2) * kTcDrainCols;
        const uint32_t tbase = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
        for (int t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
            const TcTile tl = tc_tile(t, per_item, TC, sym);
            const bool live = c0 < tc_tile_n(n, tl.col0);  // this warp's columns hold results
            const int rbase = tl.row0 + (warp & 3) * 32, cbase = tl.col0 + c0;
            const bool work = live && rbase < n;  // warp-uniform
            // the exponents of the row (this lane's) and of column cbase + lane % 16,
            // loaded before the accumulators are ready; past n a valid column's
            int er = 0, ecl = 0;
            if (work) {
                if (rbase + lane < n) er = ea_all[(size_t)(tl.b % a_mod) * n + rbase + lane];
                const int cl = cbase + (lane & 15);
                ecl = eb_all[(size_t)tl.b * n + (cl < n ? cl : cbase)];
            }
            long long acc[kTcDrainCols];
#pragma unroll
            for (int j = 0; j < kTcDrainCols; ++j) acc[j] = 0;
            for (int k0 = 0; k0 < Kp; k0 += kTcKBlk, ++blk) {
                if (!__all_sync(0xffffffffu, tc_wait(accf_s, (uint32_t)(blk & 1), abort_flag))) {
                    failed = true;
                    break;
                }
                tc_fence_after();
                // two accumulators per round trip; the arrival that hands the tensor memory
                // back comes as soon as the last pair is in registers, so its conversion
                // runs beside the next block's MMAs
#pragma unroll
                for (int d = 0; d < kOzDigits; d += 2) {
                    uint32_t r0[kTcDrainCols], r1[kTcDrainCols];
                    const bool any = live && d <= dmax, two = any && d + 1 <= dmax;  // warp-uniform
                    if (any) tc_ld16(tbase + (uint32_t)(d * kTcN), r0);
                    if (two) tc_ld16(tbase + (uint32_t)((d + 1) * kTcN), r1);
                    if (any) tc_wait_ld();
                    const bool last = !any || d + 2 > dmax;
                    if (last) {
                        tc_fence_before();
                        mbar_arrive(acce_s);  // the tensor core may overwrite the accumulators
                    }
                    const int sh0 = 36 - 8 * d, sh1 = sh0 - 8;  // weight 2^{-8(d+2)+2} = 2^{sh-50}
                    if (any) {
#pragma unroll
                        for (int j = 0; j < kTcDrainCols; ++j) {
                            const int v = __float2int_rn(__uint_as_float(r0[j]));
                            acc[j] += sh0 >= 0 ? ((long long)v << sh0) : (long long)(v >> -sh0);
                        }
                    }
                    if (two) {
#pragma unroll
                        for (int j = 0; j < kTcDrainCols; ++j) {
                            const int v = __float2int_rn(__uint_as_float(r1[j]));
                            acc[j] += sh1 >= 0 ? ((long long)v << sh1) : (long long)(v >> -sh1);
                        }
                    }
                    if (last) break;
                }
            }
            if (failed) break;
            if (!work) continue;
            // element (r, cbase + j) = acc[j] 2^{er + ec_j - 50}: first the integers as
            // doubles of their own scale, then the exponents added to the fields
            double *C = C_all + (size_t)tl.b * n * n;
            const int r = rbase + lane;
            double v[kTcDrainCols];
            unsigned long long u[kTcDrainCols];
#pragma unroll
            for (int j = 0; j < kTcDrainCols; ++j) u[j] = i64_to_f64_bits(acc[j]);
            int emin = ecl, emax = ecl;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
                emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
            }
            if (__all_sync(0xffffffffu, er - 50 + emin >= -1022 && er - 50 + emax <= 959)) {
#pragma unroll
                for (int j = 0; j < kTcDrainCols; ++j) {
                    const long long e = er + __shfl_sync(0xffffffffu, ecl, j) - 50;
                    v[j] = __longlong_as_double(u[j] == 0 ? 0ll : (long long)(u[j] + ((unsigned long long)e << 52)));
                }
            } else {
#pragma unroll
                for (int j = 0; j < kTcDrainCols; ++j) {
                    const int e = er + __shfl_sync(0xffffffffu, ecl, j) - 50;
                    v[j] = f64_times_pow2_slow(__longlong_as_double((long long)u[j]), e);
                }
            }
            if (sym) {
                // mirrored elements C[c][r], c > r: lanes run along r, coalesced
#pragma unroll
                for (int j = 0; j < kTcDrainCols; ++j) {
                    const int c = cbase + j;
                    if (c < n && r < n && c > r) C[(size_t)c * n + r] = v[j];
                }
            }
            // lane l now takes column cbase + l % 16 of rows rg + j: each store
            // writes two 128-byte row segments
            tc_transpose16(v, lane);
            const int c = cbase + (lane & 15), rg = rbase + (lane & 16);
#pragma unroll
            for (int j = 0; j < kTcDrainCols; ++j) {
                const int rr = rg + j;
                if (rr < n && c < n && (!sym || c >= rr)) C[(size_t)rr * n + c] = v[j];
            }
        }
        if (failed) *abort_flag = 1;
    }
    if (failed) record_error(err, kDevTimeout);
    tc_fence_before();
    __syncthreads();
    if (warp == kTcMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
    }
}

static PFN_cuTensorMapEncodeTiled_v12000 tc_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3-D map of a slice set S[items][6][n][Kp] (bf16): box of kTcKC k x rows x all six digits.
static bool tc_map(CUtensorMap *m, const __nv_bfloat16 *S, int n, int Kp, int items, int rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tc_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)n, (cuuint64_t)kOzDigits * items};
    const cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)n * Kp * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kTcKC, (cuuint32_t)rows, (cuuint32_t)kOzDigits};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(S), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// a_items: the number of A slice sets; item b multiplies A set b % a_items (a_items =
// items: one A per item; a_items < items: A sets shared cyclically, e.g. one per
// channel of a bucket whose items run channel-fastest).
cudaError_t launch_oz_gemm_tc(int n, int items, const __nv_bfloat16 *sa, const int *ea, const __nv_bfloat16 *sb,
                              const int *eb, double *C, int digits, bool sym, int *err, cudaStream_t st, int a_items)
{
    if (a_items <= 0) a_items = items;
    if (n < 1 || items < 1 || digits < 1 || digits > kOzDigits || a_items > items) return cudaErrorInvalidValue;
    const int Kp = oz_kpad(n);
    if (Kp % kTcKC != 0) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!tc_map(&ma, sa, n, Kp, a_items, kTcM) || !tc_map(&mb, sb, n, Kp, items, kTcN)) return cudaErrorInvalidValue;
    const int TR = (n + kTcM - 1) / kTcM, TC = (n + kTcN - 1) / kTcN;
    int per_item = TR * TC;
    if (sym) {
        per_item = 0;
        for (int tr = 0; tr < TR; ++tr) per_item += TC - 2 * tr;  // >= 1 for every tr < TR
    }
    const long long ntiles = (long long)per_item * items;
    if (ntiles > 0x7fffffffll) return cudaErrorInvalidValue;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    cudaError_t e = cudaFuncSetAttribute(k_oz_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    k_oz_gemm_tc<<<grid, kTcThreads, kTcSmem, counted(st)>>>(ma, mb, n, Kp, digits - 1, sym, per_item, TC, (int)ntiles, ea, eb,
                                                    C, err, a_items);
    return cudaGetLastError();
}

}  // namespace wpcd
