// Split-precision GEMM on the fifth-generation tensor cores (tcgen05).
//
// C = alpha op(A) op(B) + beta C with FP64 inputs and output.  Each operand is
// split into a TF32 head and a TF32 tail, x = hi + lo with hi = tf32(x) and
// lo = tf32(x - hi) (|x - hi - lo| <= 2^-22 |x|), and the product is taken as
//     hi_A hi_B  +  (hi_A lo_B + lo_A hi_B)
// on the tensor cores (the dropped lo_A lo_B term is 2^-22 relative).  The
// BF16 variant splits into bfloat16 head and tail the same way (2^-16).
//
// Accumulation.  A tensor-core FP32 accumulator that runs over the whole K
// loses about one unit in the last place per accumulation step, which over
// K = 1024 is ~1e-5 relative.  Here every 128-byte K block (32 TF32 or 64
// BF16 terms) starts fresh accumulators in tensor memory, one for the head
// product and one for the two correction products, and the epilogue warps
// add each finished block into double-float (hi + lo FP32 pair, TwoSum)
// registers while the tensor cores work on the next block.  Tensor memory
// holds two such accumulator pairs (double buffering).
//
// Roles in one CTA (one 128 x 64 tile of C, 160 threads):
//   * warp 4, lane 0: TMA loads of 128-byte K slices (128-byte swizzle) into a
//     4-deep ring of shared-memory stages, each guarded by an mbarrier that
//     counts the landed bytes; tcgen05.mma of the three products per 32-byte
//     K step; tcgen05.commit to release the stage and to publish the
//     accumulator buffer;
//   * warps 0-3: wait for a published buffer, read it with tcgen05.ld (warp w
//     owns TMEM lanes 32w..32w+31 = rows of the tile), accumulate, hand the
//     buffer back through an mbarrier; finally write alpha acc + beta C.
// Every mbarrier wait is bounded (about one second of device time); on expiry
// the kernel records an error in g_tc_status, drains its own outstanding TMA
// loads (again bounded), frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <algorithm>
#include "common.cuh"
#include "kernels.cuh"

namespace tn {

static __device__ int g_tc_status;     // 0 = fine, else a wait expired in a tensor-core kernel

namespace {

constexpr int BM = 128;                 // rows of a C tile = UMMA M = TMEM lanes
constexpr uint32_t ROWB = 128;          // bytes of K per operand row and stage (one swizzle row)
constexpr unsigned long long WAIT_NS = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(a), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(a) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete; false after WAIT_NS.
__device__ bool mbar_wait(uint32_t a, uint32_t parity)
{
    if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try(a, parity))
        if (gtimer() - t0 > WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 :: "r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int KIND>
__device__ __forceinline__ void tc_mma(uint32_t d, unsigned long long a, unsigned long long b, uint32_t idesc,
                                       uint32_t acc)
{
    if constexpr (KIND == 0) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
    } else {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                     :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
    }
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(bar) : "memory");
}

// 16 consecutive 32-bit columns of the warp's 32 TMEM lanes (one row per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte
// swizzled layout written by TMA: rows of 128 bytes, 8-row groups 1024 bytes
// apart (stride byte offset), leading byte offset unused for this layout,
// descriptor version 1, swizzle mode 2 (128 bytes).  The tile base is 1024-byte
// aligned; a K step inside the swizzle row advances the start address.
__device__ __forceinline__ unsigned long long smem_desc(uint32_t saddr)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((saddr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)1 << 16;                    // leading byte offset (16 B, ignored)
    d |= (unsigned long long)(1024u >> 4) << 32;         // stride byte offset
    d |= (unsigned long long)1 << 46;                    // descriptor version
    d |= (unsigned long long)2 << 61;                    // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulator, A and B of the kind's type, both
// K-major, N = bn, M = 128.
template <int KIND>
__host__ __device__ constexpr uint32_t instr_desc(int bn)
{
    return (1u << 4)                                          // D format: F32
         | ((KIND == 0 ? 2u : 1u) << 7)                       // A format: TF32 / BF16
         | ((KIND == 0 ? 2u : 1u) << 10)                      // B format
         | ((uint32_t)(bn >> 3) << 17)                        // N >> 3
         | ((uint32_t)(BM >> 4) << 24);                       // M >> 4
}

constexpr int BN = 64;                  // columns of a C tile = UMMA N
constexpr int STAGES = 4;
constexpr uint32_t A_BYTES = BM * ROWB, B_BYTES = BN * ROWB;
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;     // hi and lo of both operands
constexpr uint32_t TMEM_COLS = 4 * BN;                          // 2 buffers x (head, correction)
constexpr int THREADS = 160;                                    // 4 epilogue warps + 1 issuing warp
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 + 256;

// s + x as an unevaluated FP32 pair (Knuth's TwoSum), lo collecting the rounding error.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo += err;
}

template <int KIND>
__global__ void __launch_bounds__(THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               int Mp, int Np, int nkb, int M, int N, double alpha, double beta, double* __restrict__ C,
               int ldc)
{
    constexpr int KEL = KIND == 0 ? 32 : 64;            // K elements per 128-byte row
    constexpr uint32_t IDESC = instr_desc<KIND>(BN);

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // barriers: full[STAGES], empty[STAGES], tfull[2], tfree[2]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * STAGES;
    const uint32_t tfull0 = empty0 + 8 * STAGES, tfree0 = tfull0 + 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(full0 + 8 * s, 1); mbar_init(empty0 + 8 * s, 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(tfull0 + 8 * b, 1); mbar_init(tfree0 + 8 * b, 128); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 4) {
        if (lane == 0) {
            auto load = [&](int kb) {
                const int s = kb % STAGES;
                const uint32_t st = sbase + s * STAGE_BYTES, bar = full0 + 8 * s;
                mbar_expect_tx(bar, STAGE_BYTES);
                tma_load_2d(st, &mapA, kb * KEL, m0, bar);
                tma_load_2d(st + A_BYTES, &mapA, kb * KEL, Mp + m0, bar);
                tma_load_2d(st + 2 * A_BYTES, &mapB, kb * KEL, n0, bar);
                tma_load_2d(st + 2 * A_BYTES + B_BYTES, &mapB, kb * KEL, Np + n0, bar);
            };
            bool ok = true;
            int issued = 0, kb = 0;
            for (; issued < STAGES && issued < nkb; ++issued) load(issued);
            for (; kb < nkb; ++kb) {
                const int s = kb % STAGES, b = kb & 1;
                if (kb >= 2 && !mbar_wait(tfree0 + 8 * b, ((kb >> 1) - 1) & 1)) { ok = false; break; }
                if (!mbar_wait(full0 + 8 * s, (kb / STAGES) & 1)) { ok = false; break; }
                tc_fence_after();
                const uint32_t st = sbase + s * STAGE_BYTES;
                const unsigned long long ah = smem_desc(st), al = smem_desc(st + A_BYTES);
                const unsigned long long bh = smem_desc(st + 2 * A_BYTES), bl = smem_desc(st + 2 * A_BYTES + B_BYTES);
                const uint32_t t_head = tmem + (uint32_t)(b * 2 * BN), t_corr = t_head + BN;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {                 // 32 bytes of K per product
                    const unsigned long long o = (unsigned long long)(ks * 2);   // 32 B >> 4
                    tc_mma<KIND>(t_head, ah + o, bh + o, IDESC, ks != 0);
                    tc_mma<KIND>(t_corr, ah + o, bl + o, IDESC, ks != 0);
                    tc_mma<KIND>(t_corr, al + o, bh + o, IDESC, 1);
                }
                tc_commit(empty0 + 8 * s);
                tc_commit(tfull0 + 8 * b);
                if (kb >= 1 && issued < nkb) {                   // refill the stage k-block kb-1 used
                    const int sp = (kb - 1) % STAGES;
                    if (!mbar_wait(empty0 + 8 * sp, ((kb - 1) / STAGES) & 1)) { ok = false; ++kb; break; }
                    load(issued);
                    ++issued;
                }
            }
            if (!ok) {
                for (int j = kb; j < issued; ++j) mbar_wait(full0 + 8 * (j % STAGES), (j / STAGES) & 1);
                atomicExch(&g_tc_status, 1);
            }
        }
        __syncwarp();
    } else {
        // epilogue warps: row of the tile = TMEM lane
        float acc_hi[BN], acc_lo[BN];
#pragma unroll
        for (int j = 0; j < BN; ++j) { acc_hi[j] = 0.0f; acc_lo[j] = 0.0f; }
        const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb) {
            const int b = kb & 1;
            if (!mbar_wait(tfull0 + 8 * b, (kb >> 1) & 1)) ok = false;
            ok = __all_sync(0xffffffffu, ok);        // warp-uniform: tcgen05.ld is warp-collective
            tc_fence_after();
            const uint32_t t_head = tmem + lane_off + (uint32_t)(b * 2 * BN), t_corr = t_head + BN;
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t h[16], c[16];
                tmem_ld16(t_head + (uint32_t)c0, h);
                tmem_ld16(t_corr + (uint32_t)c0, c);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    two_sum_acc(acc_hi[c0 + j], acc_lo[c0 + j], __uint_as_float(h[j]));
                    acc_lo[c0 + j] += __uint_as_float(c[j]);
                }
            }
            tc_fence_before();
            mbar_arrive(tfree0 + 8 * b);
            if (!ok) break;
        }
        if (!ok) atomicExch(&g_tc_status, 2);
        const int row = m0 + warp * 32 + lane;
        if (row < M) {
            double* crow = C + (size_t)row * ldc;
#pragma unroll
            for (int j = 0; j < BN; ++j) {
                const int col = n0 + j;
                if (col < N) {
                    double v = alpha * ((double)acc_hi[j] + (double)acc_lo[j]);
                    if (beta != 0.0) v += beta * crow[col];
                    crow[col] = v;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------------------
// operand split: FP64 -> head/tail of the tensor-core type, K-major, padded
// ---------------------------------------------------------------------------
__device__ __forceinline__ float tf32_rn(float f)
{
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7f800000u) != 0x7f800000u) u += 0xfffu + ((u >> 13) & 1u);   // round to nearest even
    return __uint_as_float(u & 0xffffe000u);
}

__device__ __forceinline__ void split_store(float* out, size_t hi_at, size_t lo_at, double x)
{
    const float h = tf32_rn((float)x);
    out[hi_at] = h;
    out[lo_at] = tf32_rn((float)(x - (double)h));
}

__device__ __forceinline__ void split_store(__nv_bfloat16* out, size_t hi_at, size_t lo_at, double x)
{
    const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
    out[hi_at] = h;
    out[lo_at] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
}

// Logical operand X (R x K): element (r, k) at X[r*ld + k] when kcontig, else
// at X[k*ld + r].  Output rows r < Rp: hi at out[r*Kp + k], lo at
// out[(Rp + r)*Kp + k]; zero outside R x K.  32 x 32 tiles, 32 x 8 threads.
template <typename T>
__global__ void split_kernel(const double* __restrict__ X, int ld, int kcontig, int R, int K, int Rp, int Kp,
                             T* __restrict__ out)
{
    __shared__ double tile[32][33];
    const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (kcontig) {
        for (int i = ty; i < 32; i += 8) {
            const int r = r0 + i, k = k0 + tx;
            tile[i][tx] = (r < R && k < K) ? X[(size_t)r * ld + k] : 0.0;
        }
    } else {
        for (int i = ty; i < 32; i += 8) {
            const int k = k0 + i, r = r0 + tx;
            tile[tx][i] = (r < R && k < K) ? X[(size_t)k * ld + r] : 0.0;
        }
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int r = r0 + i, k = k0 + tx;
        split_store(out, (size_t)r * Kp + k, (size_t)(Rp + r) * Kp + k, tile[i][tx]);
    }
}

// ---------------------------------------------------------------------------
// Exact-accumulation slices (the Ozaki scheme: Ozaki, Ogita, Oishi, Rump,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Row i of op(A) is scaled by 2^-e_i, e_i the binary exponent of its largest
// |entry| (so every scaled entry lies in (-1, 1)), and cut into S slices of
// 8 bits by truncation:  A_ik = 2^e_i sum_{s<S} a^(s)_ik 2^-8(s+1) + r_ik, the
// a^(s) integers in [0, 255] carrying the sign of A_ik (exact in BF16, which
// holds 8 significant bits), |r_ik| < 2^(e_i - 8S); likewise the columns of
// op(B) with exponents f_j.  The product keeps the levels L = s + t < S,
//     C_ij = 2^(e_i + f_j - 16) sum_{L<S} 2^-8L  P_L,   P_L = sum_{s+t=L} a^(s) b^(t)
// (S (S+1) / 2 slice products).  Every product of two slices is an integer of
// magnitude below 2^16, and level L (L + 1 products) summed over one K block of
// KROW elements stays below (L + 1) KROW 255^2 < 2^24 (4 slices, KROW = 64,
// level 3: 16 646 400; 7 slices, KROW = 32, level 6: 14 565 600): the FP32
// tensor-core accumulator holds it exactly, whatever its rounding.  Each block's
// level sums are read from tensor memory, converted to integers (exact) and
// added into 64-bit integers, levels 0..H-1 into one and the rest into a second,
//     Q_0 += sum_{L<H} P_L 2^8(H-1-L),   Q_1 += sum_{L>=H} P_L 2^8(S-1-L),
// so the only roundings are the final conversions of Q_0, Q_1 to double (exact
// while they stay below 2^53: for K <= 8192 with 4 slices, K <= 2048 for Q_1
// with 7 slices; beyond, a rounding at the FP64 unit roundoff of the partial
// sum).  The dropped levels L >= S (all pairs s + t = L, slices beyond S
// included) leave, per term of the K sum, at most
//     2^(e_i + f_j) 255^2 2^-16 sum_{L>=S} (L + 1) 2^-8L  <  (S + 1) 2^-8S 2^(e_i + f_j),
// and 2^(e_i + f_j) <= 4 max|A_i.| max|B_.j|, so
//     |C - AB|_ij < 4 (S + 1) 2^-8S K max|A_i.| max|B_.j|
// (4 slices: 20 * 2^-32 ~ 2^-27.7; 7 slices: 32 * 2^-56 = 2^-51, the FP64 unit
// roundoff level of a K-term sum).  On Gaussian operands the per-term errors
// partly cancel, ~1e-9 relative (4 slices).
// ---------------------------------------------------------------------------
// Two configurations: 4 slices (10 products) for the precision form, and 7
// slices (28 products) for FP64-accurate products.  A K block of KROW elements
// is one shared-memory row per operand row (128-byte rows with 128-byte swizzle
// for 4 slices, 64-byte rows with 64-byte swizzle for 7, so that three stages
// fit) and is drained after every K block.  H = 4 for 4 slices (one integer),
// H = 3 for 7 slices.
template <int S> struct OzCfg;
template <> struct OzCfg<4> {
    static constexpr int BN = 64, KROW = 64, STAGES = 2, H = 4, SWZ = 2;    // 128-byte swizzle
};
template <> struct OzCfg<7> {
    static constexpr int BN = 32, KROW = 32, STAGES = 3, H = 3, SWZ = 4;    // 64-byte swizzle
};
constexpr int OZ_PRODUCER = 8;                                 // warps 0-7 drain tensor memory
constexpr int OZ_THREADS = 32 * (OZ_PRODUCER + 1);

template <int S>
struct OzLayout {
    using C = OzCfg<S>;
    static constexpr uint32_t ROW = C::KROW * 2;                           // bytes per operand row per stage
    static constexpr uint32_t A_BYTES = S * BM * ROW, B_BYTES = S * C::BN * ROW;
    static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr uint32_t COLS_USED = 2 * S * C::BN;                  // 2 buffers x S levels
    static constexpr uint32_t TMEM_COLS = COLS_USED <= 256 ? 256 : 512;
    static constexpr size_t SMEM = (size_t)C::STAGES * STAGE_BYTES + 1024 + 256;
};

// Shared-memory descriptor of a K-major tile with `swz` swizzle (2: 128-byte rows,
// 4: 64-byte rows); 8-row groups are 8 rows apart (stride byte offset).
__device__ __forceinline__ unsigned long long smem_desc_sw(uint32_t saddr, uint32_t row_bytes, uint32_t swz)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((saddr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)1 << 16;                              // leading byte offset (ignored)
    d |= (unsigned long long)((8u * row_bytes) >> 4) << 32;        // stride byte offset
    d |= (unsigned long long)1 << 46;                              // descriptor version
    d |= (unsigned long long)swz << 61;
    return d;
}

// C (or the partial product of K-split z into P) from the slices; grid
// (Np / BN, Mp / BM, splits).
template <int S>
__global__ void __launch_bounds__(OZ_THREADS, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               int Mp, int Np, int nkb, int M, int N, const int* __restrict__ ea, const int* __restrict__ fb,
               double alpha, double beta, double* __restrict__ C, int ldc, double* __restrict__ P)
{
    using Cf = OzCfg<S>;
    using Ly = OzLayout<S>;
    constexpr int BNs = Cf::BN, KEL = Cf::KROW, NST = Cf::STAGES, H = Cf::H;
    constexpr uint32_t IDESC = instr_desc<1>(BNs);

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NST * Ly::STAGE_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * NST + 4);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * NST;
    const uint32_t tfull0 = empty0 + 8 * NST, tfree0 = tfull0 + 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BNs;
    // this CTA's K blocks (K split over blockIdx.z)
    const int kb0 = (int)(((long long)nkb * blockIdx.z) / gridDim.z);
    const int kb1 = (int)(((long long)nkb * (blockIdx.z + 1)) / gridDim.z);
    const int nk = kb1 - kb0;

    if (warp == OZ_PRODUCER) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(Ly::TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) { mbar_init(full0 + 8 * s, 1); mbar_init(empty0 + 8 * s, 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(tfull0 + 8 * b, 1); mbar_init(tfree0 + 8 * b, 32 * OZ_PRODUCER); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == OZ_PRODUCER) {
        if (lane == 0) {
            auto load = [&](int j) {
                const int s = j % NST;
                const uint32_t st = sbase + s * Ly::STAGE_BYTES, bar = full0 + 8 * s;
                mbar_expect_tx(bar, Ly::STAGE_BYTES);
                for (int q = 0; q < S; ++q) tma_load_2d(st + q * BM * Ly::ROW, &mapA, (kb0 + j) * KEL, q * Mp + m0, bar);
                for (int q = 0; q < S; ++q)
                    tma_load_2d(st + Ly::A_BYTES + q * BNs * Ly::ROW, &mapB, (kb0 + j) * KEL, q * Np + n0, bar);
            };
            bool ok = true;
            int issued = 0, kb = 0;
            for (; issued < NST && issued < nk; ++issued) load(issued);
            for (; kb < nk; ++kb) {
                const int s = kb % NST, b = kb & 1;
                if (kb >= 2 && !mbar_wait(tfree0 + 8 * b, ((kb >> 1) - 1) & 1)) { ok = false; break; }
                if (!mbar_wait(full0 + 8 * s, (kb / NST) & 1)) { ok = false; break; }
                tc_fence_after();
                const uint32_t st = sbase + s * Ly::STAGE_BYTES;
                const uint32_t tb = tmem + (uint32_t)(b * S * BNs);
#pragma unroll
                for (int ks = 0; ks < KEL / 16; ++ks) {          // 16 bf16 of K (32 bytes) per product
                    const unsigned long long o = (unsigned long long)(ks * 2);
#pragma unroll
                    for (int L = 0; L < S; ++L)
#pragma unroll
                        for (int sa = 0; sa <= L; ++sa) {
                            const int sb = L - sa;
                            const unsigned long long da = smem_desc_sw(st + sa * BM * Ly::ROW, Ly::ROW, Cf::SWZ) + o;
                            const unsigned long long db =
                                smem_desc_sw(st + Ly::A_BYTES + sb * BNs * Ly::ROW, Ly::ROW, Cf::SWZ) + o;
                            tc_mma<1>(tb + (uint32_t)(L * BNs), da, db, IDESC, (ks != 0 || sa != 0) ? 1u : 0u);
                        }
                }
                tc_commit(empty0 + 8 * s);
                tc_commit(tfull0 + 8 * b);
                if (kb >= 1 && issued < nk) {                    // refill the stage k-block kb-1 used
                    const int sp = (kb - 1) % NST;
                    if (!mbar_wait(empty0 + 8 * sp, ((kb - 1) / NST) & 1)) { ok = false; ++kb; break; }
                    load(issued);
                    ++issued;
                }
            }
            if (!ok) {
                for (int j = kb; j < issued; ++j) mbar_wait(full0 + 8 * (j % NST), (j / NST) & 1);
                atomicExch(&g_tc_status, 1);
            }
        }
        __syncwarp();
    } else {
        // epilogue warp w: TMEM lanes 32 (w % 4) .. + 31 (the rows of the tile it may read)
        // and the half (w / 4) of the tile's columns
        constexpr int HC = BNs / 2;
        constexpr int NACC = (H < S) ? 2 : 1;
        const int cbase = (warp >> 2) * HC;
        long long acc[NACC][HC];
#pragma unroll
        for (int a = 0; a < NACC; ++a)
#pragma unroll
            for (int j = 0; j < HC; ++j) acc[a][j] = 0;
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb) {
            const int b = kb & 1;
            if (!mbar_wait(tfull0 + 8 * b, (kb >> 1) & 1)) ok = false;
            ok = __all_sync(0xffffffffu, ok);        // warp-uniform: tcgen05.ld is warp-collective
            tc_fence_after();
            const uint32_t tb = tmem + lane_off + (uint32_t)(b * S * BNs + cbase);
#pragma unroll
            for (int c0 = 0; c0 < HC; c0 += 16) {
#pragma unroll
                for (int L = 0; L < S; ++L) {
                    uint32_t p[16];
                    tmem_ld16(tb + (uint32_t)(L * BNs + c0), p);
                    const int a = L < H ? 0 : 1;
                    const int sh = L < H ? 8 * (H - 1 - L) : 8 * (S - 1 - L);
#pragma unroll
                    for (int j = 0; j < 16; ++j)    // exact integers below 2^24: exact conversions
                        acc[a < NACC ? a : 0][c0 + j] += (long long)__float2int_rn(__uint_as_float(p[j])) * (1LL << sh);
                }
            }
            tc_fence_before();
            mbar_arrive(tfree0 + 8 * b);
            if (!ok) break;
        }
        if (!ok) atomicExch(&g_tc_status, 2);
        const int row = m0 + (warp & 3) * 32 + lane;
        if (row < M) {
            // 2^(e_i + f_j - 16) times the level weights; rows or columns of zeros carry a
            // huge negative exponent (their sums are 0): clamp it so the sum cannot overflow
            const int er = max(ea[row], -4000) - 16;
#pragma unroll
            for (int j = 0; j < HC; ++j) {
                const int col = n0 + cbase + j;
                if (col < N) {
                    const int ex = er + max(fb[col], -4000);
                    double v = ldexp((double)acc[0][j], ex - 8 * (H - 1));
                    if (NACC == 2) v += ldexp((double)acc[NACC - 1][j], ex - 8 * (S - 1));
                    if (P) {
                        P[((size_t)blockIdx.z * M + row) * N + col] = v;
                    } else {
                        double* dst = C + (size_t)row * ldc + col;
                        *dst = (beta == 0.0) ? alpha * v : alpha * v + beta * (*dst);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == OZ_PRODUCER)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(Ly::TMEM_COLS) : "memory");
}

// C = alpha sum_z P[z] + beta C (K-split partial products, summed in split order)
__global__ void oz_reduce_kernel(const double* __restrict__ P, int splits, int M, int N, double alpha, double beta,
                                 double* __restrict__ C, int ldc)
{
    const long long mn = (long long)M * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mn; e += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int z = 0; z < splits; ++z) acc += P[z * mn + e];
        const int r = (int)(e / N), c = (int)(e % N);
        double* dst = C + (size_t)r * ldc + c;
        *dst = (beta == 0.0) ? alpha * acc : alpha * acc + beta * (*dst);
    }
}

// Binary exponent of max |entry| of every row r of the logical operand X (R x K,
// layout as split_kernel): e[r] = the e with max < 2^e (frexp), atomically
// maximised over tiles; e must start at OZ_EMPTY.  Rows of zeros keep OZ_EMPTY.
constexpr int OZ_EMPTY = -100000;

__global__ void oz_exponent_kernel(const double* __restrict__ X, int ld, int kcontig, int R, int K, int* __restrict__ e)
{
    __shared__ int red[32][33];
    const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    // element (r0 + i, k0 + j) goes to red[i][j]
    for (int i = ty; i < 32; i += 8) {
        int r, k;
        double x;
        if (kcontig) { r = r0 + i; k = k0 + tx; x = (r < R && k < K) ? X[(size_t)r * ld + k] : 0.0; }
        else { k = k0 + i; r = r0 + tx; x = (r < R && k < K) ? X[(size_t)k * ld + r] : 0.0; }
        // the frexp exponent (x = f 2^ex, 1/2 <= |f| < 1) from the bits: x = m 2^e2 with
        // significand m, ex = bitlength(m) + e2 (integer arithmetic, subnormals included)
        int ex = OZ_EMPTY;
        if (x != 0.0) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
            const int bexp = (int)(u >> 52);
            const unsigned long long m = (u & 0x000fffffffffffffull) | (bexp ? 0x0010000000000000ull : 0ull);
            ex = (64 - __clzll((long long)m)) + (bexp ? bexp : 1) - 1075;
        }
        if (kcontig) red[i][tx] = ex; else red[tx][i] = ex;
    }
    __syncthreads();
    if (ty == 0) {
        int m = OZ_EMPTY;
        for (int j = 0; j < 32; ++j) m = max(m, red[tx][j]);
        if (r0 + tx < R && m > OZ_EMPTY) atomicMax(&e[r0 + tx], m);
    }
}

// Slices of the scaled operand: out[(q * Rp + r) * Kp + k] = a^(q)_rk (BF16 integers),
// zero outside R x K and for rows of zeros.
template <int S>
__global__ void oz_slice_kernel(const double* __restrict__ X, int ld, int kcontig, int R, int K, int Rp, int Kp,
                                const int* __restrict__ e, __nv_bfloat16* __restrict__ out)
{
    __shared__ double tile[32][33];
    const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (kcontig) {
        for (int i = ty; i < 32; i += 8) {
            const int r = r0 + i, k = k0 + tx;
            tile[i][tx] = (r < R && k < K) ? X[(size_t)r * ld + k] : 0.0;
        }
    } else {
        for (int i = ty; i < 32; i += 8) {
            const int k = k0 + i, r = r0 + tx;
            tile[tx][i] = (r < R && k < K) ? X[(size_t)k * ld + r] : 0.0;
        }
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int r = r0 + i, k = k0 + tx;
        const int er = (r < R) ? e[r] : OZ_EMPTY;
        const double x = tile[i][tx];
        // |v| = |x| 2^-er < 1 as the fixed-point integer F = floor(|v| 2^(8S)) (at most 56 bits),
        // read off the binary representation: x = m 2^e2 with the 53-bit significand m.  The
        // slices are F's bytes from the top, with the sign of x: the same digits as repeated
        // "times 256, truncate, keep the remainder" in FP64, without FP64 arithmetic (the
        // FP64 pipe, 1/64 of FP32 on this GPU, made that the slowest pass of the product).
        unsigned long long F = 0;
        if (er > OZ_EMPTY && x != 0.0) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
            const int bexp = (int)(u >> 52);
            const unsigned long long m = (u & 0x000fffffffffffffull) | (bexp ? 0x0010000000000000ull : 0ull);
            const int sh = (bexp ? bexp : 1) - 1075 + 8 * S - er;          // F = floor(m 2^sh)
            F = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);  // m 2^sh < 2^(8S): no overflow
        }
        const bool neg = x < 0.0;
        for (int q = 0; q < S; ++q) {
            const int a = (int)((F >> (8 * (S - 1 - q))) & 0xffull);     // integer in [0, 255]
            out[((size_t)q * Rp + r) * Kp + k] = __float2bfloat16_rn((float)(neg ? -a : a));   // exact
        }
    }
}

// The driver's tensor-map encoder, looked up once (a function-local static is
// initialised exactly once even when several host threads get here first).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

int encoder() { return encode_fn() ? TN_OK : TN_ECUDA; }

// 2D map over a rows2 x Kp operand buffer, box = row_bytes of K x box_rows, with the
// swizzle that matches row_bytes (128 or 64 bytes).
int make_map(CUtensorMap* map, int kind, void* base, int rows2, int Kp, int box_rows, int row_bytes = (int)ROWB)
{
    const int esz = kind == 0 ? 4 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows2};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * esz};
    cuuint32_t box[2] = {(cuuint32_t)(row_bytes / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(map, kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                          base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? TN_OK : TN_ECUDA;
}

template <int KIND>
int launch_tc(cudaStream_t st, const CUtensorMap& ma, const CUtensorMap& mb, int Mp, int Np, int nkb, int m, int n,
              double alpha, double beta, double* C, int ldc)
{
    static std::atomic<unsigned long long> attr{0};
    TN_CUDA(tn_smem_optin(tc_gemm_kernel<KIND>, (int)SMEM_BYTES, attr));
    dim3 grid(Np / BN, Mp / BM);
    tc_gemm_kernel<KIND><<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, Mp, Np, nkb, m, n, alpha, beta, C, ldc);
    TN_LAUNCHED();
    return TN_OK;
}

inline int round_up(int x, int q) { return (x + q - 1) / q * q; }

// Tile and K-split plan of a slice product.
struct OzPlan { int Mp, Np, Kp, nkb, splits; };

template <int S>
OzPlan oz_plan(int m, int n, int k)
{
    using Cf = OzCfg<S>;
    OzPlan p;
    p.Mp = round_up(m, BM);
    p.Np = round_up(n, Cf::BN);
    p.Kp = round_up(k, Cf::KROW);
    p.nkb = p.Kp / Cf::KROW;
    const int tiles = (p.Mp / BM) * (p.Np / Cf::BN);
    // products with few tiles (panels, Gram blocks) split K so that about one
    // CTA per SM is busy; every split keeps at least two K blocks
    p.splits = tiles >= 152 ? 1 : std::max(1, std::min(152 / tiles, p.nkb / 2));
    return p;
}

template <int S>
size_t oz_scratch(int m, int n, int k)
{
    const OzPlan p = oz_plan<S>(m, n, k);
    size_t b = tn_align256((size_t)S * p.Mp * p.Kp * 2) + tn_align256((size_t)S * p.Np * p.Kp * 2)
             + tn_align256((size_t)p.Mp * 4) + tn_align256((size_t)p.Np * 4);
    if (p.splits > 1) b += tn_align256((size_t)p.splits * m * n * 8);
    return b;
}

// Self-test of the bounded waits: one thread waits on an mbarrier that nothing
// arrives on, with the wait the tensor-core kernels use.  The wait expires
// after WAIT_NS, the kernel records the expiry in g_tc_status (value 3) and
// returns; no TMA copy or tensor memory is involved.
__global__ void wait_probe_kernel()
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        const uint32_t a = smem_u32(&bar);
        mbar_init(a, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait(a, 0)) atomicExch(&g_tc_status, 3);
    }
}

}  // namespace

int wait_selftest(cudaStream_t st, int* status)
{
    wait_probe_kernel<<<1, 32, 0, st>>>();
    TN_LAUNCHED();
    return tc_status(st, status);
}

int tc_tile_n(int, int) { return BN; }

size_t gemm_tc_scratch_bytes(int kind, int m, int n, int k)
{
    const int bn = tc_tile_n(m, n);
    if (kind == 2) return oz_scratch<4>(m, n, k);
    if (kind == 3) return oz_scratch<7>(m, n, k);
    const int kq = kind == 0 ? 32 : 64;
    const size_t esz = kind == 0 ? 4 : 2;
    const size_t Mp = round_up(m, BM), Np = round_up(n, bn), Kp = round_up(k, kq);
    return tn_align256(2 * Mp * Kp * esz) + tn_align256(2 * Np * Kp * esz);
}

// Exact-accumulation product (kinds 2 and 3): exponents, slices, one tensor-core
// pass (K split over several CTAs for products with few tiles, then a sum).
template <int S>
static int gemm_oz(cudaStream_t st, Arena& ar, bool ta, bool tb, int m, int n, int k, double alpha,
                   const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc)
{
    using Cf = OzCfg<S>;
    using Ly = OzLayout<S>;
    const OzPlan p = oz_plan<S>(m, n, k);
    const size_t mark = ar.mark();
    void* As = ar.take(((size_t)S * p.Mp * p.Kp * 2 + 7) / 8);
    void* Bs = ar.take(((size_t)S * p.Np * p.Kp * 2 + 7) / 8);
    int* ea = reinterpret_cast<int*>(ar.take(((size_t)p.Mp * 4 + 7) / 8));
    int* fb = reinterpret_cast<int*>(ar.take(((size_t)p.Np * 4 + 7) / 8));
    double* P = p.splits > 1 ? ar.take((size_t)p.splits * m * n) : nullptr;
    if (!As || !Bs || !ea || !fb || (p.splits > 1 && !P)) { ar.release(mark); return TN_ENOMEM; }
    TN_CUDA(cudaMemsetAsync(ea, 0x80, (size_t)p.Mp * 4, st));       // 0x80808080 < OZ_EMPTY
    TN_CUDA(cudaMemsetAsync(fb, 0x80, (size_t)p.Np * 4, st));
    dim3 blk(32, 8);
    // A: rows m, K-contiguous unless transposed; B: rows n, K-contiguous only when transposed
    oz_exponent_kernel<<<dim3(p.Kp / 32, p.Mp / 32), blk, 0, st>>>(A, lda, ta ? 0 : 1, m, k, ea);
    TN_LAUNCHED();
    oz_exponent_kernel<<<dim3(p.Kp / 32, p.Np / 32), blk, 0, st>>>(B, ldb, tb ? 1 : 0, n, k, fb);
    TN_LAUNCHED();
    oz_slice_kernel<S><<<dim3(p.Kp / 32, p.Mp / 32), blk, 0, st>>>(A, lda, ta ? 0 : 1, m, k, p.Mp, p.Kp, ea,
                                                                  (__nv_bfloat16*)As);
    TN_LAUNCHED();
    oz_slice_kernel<S><<<dim3(p.Kp / 32, p.Np / 32), blk, 0, st>>>(B, ldb, tb ? 1 : 0, n, k, p.Np, p.Kp, fb,
                                                                  (__nv_bfloat16*)Bs);
    TN_LAUNCHED();
    CUtensorMap ma, mb;
    int s1 = make_map(&ma, 1, As, S * p.Mp, p.Kp, BM, (int)Ly::ROW);
    int s2 = make_map(&mb, 1, Bs, S * p.Np, p.Kp, Cf::BN, (int)Ly::ROW);
    if (s1 != TN_OK || s2 != TN_OK) { ar.release(mark); return TN_ECUDA; }
    static std::atomic<unsigned long long> attr{0};
    TN_CUDA(tn_smem_optin(oz_gemm_kernel<S>, (int)Ly::SMEM, attr));
    dim3 grid(p.Np / Cf::BN, p.Mp / BM, p.splits);
    oz_gemm_kernel<S><<<grid, OZ_THREADS, Ly::SMEM, st>>>(ma, mb, p.Mp, p.Np, p.nkb, m, n, ea, fb, alpha, beta, C,
                                                          ldc, P);
    TN_LAUNCHED();
    if (P) {
        const long long mn = (long long)m * n;
        const int blocks = (int)std::min<long long>((mn + 255) / 256, 152 * 8);
        oz_reduce_kernel<<<blocks, 256, 0, st>>>(P, p.splits, m, n, alpha, beta, C, ldc);
        TN_LAUNCHED();
    }
    ar.release(mark);       // stream-ordered: later work on this stream may reuse the buffers
    return TN_OK;
}

int gemm_tc(cudaStream_t st, Arena& ar, int kind, bool ta, bool tb, int m, int n, int k, double alpha,
            const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc)
{
    if (m < 1 || n < 1 || k < 1 || kind < 0 || kind > 3) return TN_EINVAL;
    TN_TRY(encoder());
    if (kind == 2) return gemm_oz<4>(st, ar, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    if (kind == 3) return gemm_oz<7>(st, ar, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    const int bn = tc_tile_n(m, n);
    const int kq = kind == 0 ? 32 : 64;
    const size_t esz = kind == 0 ? 4 : 2;
    const int Mp = round_up(m, BM), Np = round_up(n, bn), Kp = round_up(k, kq);
    const size_t mark = ar.mark();
    void* As = ar.take((2 * (size_t)Mp * Kp * esz + 7) / 8);
    void* Bs = ar.take((2 * (size_t)Np * Kp * esz + 7) / 8);
    if (!As || !Bs) { ar.release(mark); return TN_ENOMEM; }
    // A: rows m, K-contiguous unless transposed; B: rows n, K-contiguous only when transposed
    dim3 blk(32, 8);
    if (kind == 0) {
        split_kernel<float><<<dim3(Kp / 32, Mp / 32), blk, 0, st>>>(A, lda, ta ? 0 : 1, m, k, Mp, Kp, (float*)As);
        TN_LAUNCHED();
        split_kernel<float><<<dim3(Kp / 32, Np / 32), blk, 0, st>>>(B, ldb, tb ? 1 : 0, n, k, Np, Kp, (float*)Bs);
        TN_LAUNCHED();
    } else {
        split_kernel<__nv_bfloat16><<<dim3(Kp / 32, Mp / 32), blk, 0, st>>>(A, lda, ta ? 0 : 1, m, k, Mp, Kp,
                                                                             (__nv_bfloat16*)As);
        TN_LAUNCHED();
        split_kernel<__nv_bfloat16><<<dim3(Kp / 32, Np / 32), blk, 0, st>>>(B, ldb, tb ? 1 : 0, n, k, Np, Kp,
                                                                             (__nv_bfloat16*)Bs);
        TN_LAUNCHED();
    }
    CUtensorMap ma, mb;
    int s1 = make_map(&ma, kind, As, 2 * Mp, Kp, BM);
    int s2 = make_map(&mb, kind, Bs, 2 * Np, Kp, bn);
    if (s1 != TN_OK || s2 != TN_OK) { ar.release(mark); return TN_ECUDA; }
    const int nkb = Kp / kq;
    const int s = kind == 0 ? launch_tc<0>(st, ma, mb, Mp, Np, nkb, m, n, alpha, beta, C, ldc)
                            : launch_tc<1>(st, ma, mb, Mp, Np, nkb, m, n, alpha, beta, C, ldc);
    ar.release(mark);       // stream-ordered: later work on this stream may reuse the split buffers
    return s;
}

int tc_status(cudaStream_t st, int* status)
{
    int v = 0;
    TN_CUDA(cudaMemcpyFromSymbolAsync(&v, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    TN_CUDA(cudaStreamSynchronize(st));
    *status = v;
    if (v) {
        const int zero = 0;
        TN_CUDA(cudaMemcpyToSymbolAsync(g_tc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
    }
    return TN_OK;
}

}  // namespace tn
