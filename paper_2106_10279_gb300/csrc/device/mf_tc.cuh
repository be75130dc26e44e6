// Colour sum on the tensor cores.
//
// Per helicity the colour-summed |M|^2 is sum_kl Re(conj(J_k) C_kl J_l) / den
// (the colour sum of the amplitudes, Sec. 2.4 / Fig. 1).  For the 128
// (event, helicity) rows a block holds at once this is a dense contraction:
// with A = [Re J | Im J] (128 x 2NJ) and B = diag(C, C) (2NJ x 2NJ, C real
// symmetric), Z = A B gives |M|^2_r = sum_c A_rc Z_rc / den.  Z is computed by
// tcgen05.mma (kind::tf32, M = 128) from shared-memory operands into a tensor
// memory accumulator; each thread reads its own row back (tcgen05.ld) and
// finishes the dot product on the CUDA cores with its own FP32 J.
//
// Precision: the integer numerators of C are exact in TF32.  A is split as
// A = A_hi + A_lo with A_hi = A truncated to TF32 and A_lo = A - A_hi (exact
// in FP32; the tensor core then keeps its leading 11 bits), and
// Z = A_hi B + A_lo B accumulates in FP32: each element of A enters with a
// relative error below 2^-20, close to the FP32 colour sum it replaces.
//
// Operand layout: the canonical no-swizzle K-major layout of core matrices of
// 8 rows x 16 bytes; element (r, k) of an R x KP operand sits at byte
// ((r / 8) * (KP / 4) + k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4, so that core
// matrices adjacent in K are 128 bytes apart (leading byte offset) and 8-row
// groups are KP * 32 bytes apart (stride byte offset).
//
// Every wait on the MMA's completion is bounded; on expiry the block records
// an error (the results of that round are then unspecified) and goes on, so
// that no block can hang.  Before the tensor memory is released, one more
// commit on a separate barrier tracks every MMA the block issued, and the
// block waits for it with the full limit: tensor memory is never released
// under an MMA still in flight, whatever the per-round limit was.
#pragma once
#include "mf_common.cuh"

namespace mf {
namespace tc {

constexpr int ROWS = 128;                    // rows per MMA (one per thread of a 128-thread block)
constexpr long long WAIT_LIMIT = 1ll << 24;  // polls of a completion barrier before giving up (default)

// Two operand layouts.  Side by side (2 NJ <= 128): row r of A is
// [Re J_r | Im J_r] and B = diag(C, C), one round of 128 rows per call.
// Stacked (2 NJ > 128, where diag(C, C) would not fit in shared memory):
// rows 2i and 2i+1 of A are Re J_i and Im J_i of item i and B = C; a round
// holds 64 items and a call takes two rounds (threads 0-63, then 64-127).
// Each row r then gives sum_c A_rc Z_rc, and an item's value is the sum of
// its two rows (Re(J^dagger C J) = Re J . C Re J + Im J . C Im J, C real
// symmetric).
template <int NJ>
struct Plan {
    static constexpr bool STACKED = 2 * NJ > 128;
    static constexpr int K2 = STACKED ? NJ : 2 * NJ;
    static constexpr int KP = (K2 + 7) / 8 * 8;        // K: multiple of the tf32 MMA step (8)
    static constexpr int NP = (K2 + 15) / 16 * 16;     // N: multiple of 16 for M = 128
    static constexpr int COLS = NP <= 32 ? 32 : NP <= 64 ? 64 : NP <= 128 ? 128 : 256;   // tensor-memory columns
    static constexpr int A_BYTES = ROWS * KP * 4;
    static constexpr int B_BYTES = NP * KP * 4;
    // shared-memory bytes: A_hi, A_lo, B (1 KB aligned), then the round and
    // drain barriers and the tensor-memory address; stacked: then the
    // per-thread results of a call (16-byte aligned)
    static constexpr int SMEM = STACKED ? 2 * A_BYTES + B_BYTES + 32 + ROWS * 4 : 2 * A_BYTES + B_BYTES + 24;
};

MF_DEV uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

MF_DEV uint32_t core_offset(int r, int k, int KP) {
    return (uint32_t)((((r >> 3) * (KP >> 2) + (k >> 2)) << 7) + ((r & 7) << 4) + ((k & 3) << 2));
}

// tcgen05 shared-memory matrix descriptor: start address, leading and stride
// byte offsets (all in 16-byte units), descriptor version 1, no swizzle.
MF_DEV uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32: D in f32, A and B tf32, both K-major,
// dense, N >> 3 and M >> 4.
template <int M, int N>
struct InstrDesc {
    static constexpr uint32_t value =
        (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
};

MF_DEV float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Block state: operand buffers in shared memory, the completion barrier, the
// tensor-memory base address and the barrier phase.
struct State {
    unsigned char *a_hi, *a_lo, *b;
    uint64_t *mbar;           // completion of each round's MMAs
    uint64_t *drain;          // completion of every MMA issued (teardown)
    uint32_t *tmem_slot;
    float *out;               // stacked layout: [ROWS] results of a call
    uint32_t phase;
    long long wait_limit;     // polls per round
    int *err;                 // global error flag (may be NULL)
    bool failed;
};

// Carve the buffers out of `smem` (1 KB aligned, Plan<NJ>::SMEM bytes),
// allocate tensor memory (warp 0) and initialise the barrier.  All threads.
template <int NJ>
MF_DEV void setup(State &s, unsigned char *smem, int *err, long long wait_limit = WAIT_LIMIT) {
    using P = Plan<NJ>;
    s.a_hi = smem;
    s.a_lo = smem + P::A_BYTES;
    s.b = smem + 2 * P::A_BYTES;
    s.mbar = reinterpret_cast<uint64_t *>(smem + 2 * P::A_BYTES + P::B_BYTES);
    s.drain = reinterpret_cast<uint64_t *>(smem + 2 * P::A_BYTES + P::B_BYTES + 8);
    s.tmem_slot = reinterpret_cast<uint32_t *>(smem + 2 * P::A_BYTES + P::B_BYTES + 16);
    s.out = reinterpret_cast<float *>(smem + 2 * P::A_BYTES + P::B_BYTES + 32);
    s.phase = 0;
    s.wait_limit = wait_limit < 0 ? WAIT_LIMIT : wait_limit;
    s.err = err;
    s.failed = false;
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s.tmem_slot)),
                     "r"(P::COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(s.mbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(s.drain)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Write B = diag(C, C) (integer numerators, exact in tf32), zero padded.
// All threads; a block barrier must follow before the next mma.
template <int NJ>
MF_DEV void load_colour(State &s, const int *cnum) {
    using P = Plan<NJ>;
    for (int i = threadIdx.x; i < P::NP * P::KP; i += blockDim.x) {
        const int n = i / P::KP, k = i % P::KP;
        float v = 0.f;
        if (n < NJ && k < NJ) v = (float)cnum[n * NJ + k];
        else if (!P::STACKED && n >= NJ && n < 2 * NJ && k >= NJ && k < 2 * NJ)
            v = (float)cnum[(n - NJ) * NJ + (k - NJ)];
        *reinterpret_cast<float *>(s.b + core_offset(n, k, P::KP)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

MF_DEV bool wait_phase(uint64_t *mbar, uint32_t phase, long long limit = WAIT_LIMIT) {
    const uint32_t addr = smem_u32(mbar);
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <int N>
MF_DEV void ld_cols(uint32_t taddr, float *out);

template <>
MF_DEV void ld_cols<16>(uint32_t taddr, float *out) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) out[i] = __uint_as_float(r[i]);
}

// The MMAs of one round over the operands now in A (issued by thread 0:
// Z = A_hi B + A_lo B into tensor memory), the bounded wait for them and one
// block-wide decision on its outcome.  Must be called by all 128 threads
// after they have written their rows of A.  If a round's wait expires in any
// thread, the whole block (one decision, taken at a barrier) records the
// error and from then on neither writes the operands, nor issues MMAs, nor
// reads tensor memory: its results are 0 and unspecified, and no access
// races an MMA still in flight.
template <int NJ>
MF_DEV void mma_round(State &s) {
    using P = Plan<NJ>;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s.tmem_slot;
    if (threadIdx.x == 0 && !s.failed) {
        constexpr uint32_t idesc = InstrDesc<ROWS, P::NP>::value;
        constexpr uint32_t sbo = (uint32_t)P::KP * 32;
        const uint32_t a0 = smem_u32(s.a_hi), a1 = smem_u32(s.a_lo), b0 = smem_u32(s.b);
#pragma unroll
        for (int part = 0; part < 2; ++part) {
#pragma unroll
            for (int ks = 0; ks < P::KP / 8; ++ks) {
                const uint64_t ad = smem_desc((part ? a1 : a0) + ks * 256, 128, sbo);
                const uint64_t bd = smem_desc(b0 + ks * 256, 128, sbo);
                const uint32_t acc = (part | ks) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(s.mbar))
                     : "memory");
    }
    bool ok = false;
    if (!s.failed) {
        ok = wait_phase(s.mbar, s.phase, s.wait_limit);
        s.phase ^= 1u;
    }
    // one decision for the block
    if (__syncthreads_or(!ok) && !s.failed) {
        s.failed = true;
        if (s.err && threadIdx.x == 0) atomicExch(s.err, 1);
    }
}

// The next round rewrites A and the accumulator only after every thread has
// read its row.
MF_DEV void round_done() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Stacked layout (2 NJ > 128): two rounds of 64 items; the thread reading
// row r of Z (warp r/32 reads lanes 32 (r/32) ..) takes row r of A back from
// shared memory (A_hi + A_lo is exactly the FP32 amplitude), and the two rows
// of an item, adjacent lanes of one warp, are added by a shuffle.
template <int NJ>
MF_DEV float colour_sum_stacked(State &s, const cx<float> *J) {
    using P = Plan<NJ>;
    const int t = threadIdx.x;
#pragma unroll 1
    for (int round = 0; round < 2; ++round) {
        if (!s.failed && (t >> 6) == round) {
            const int r0 = 2 * (t & 63);      // this thread's item: rows r0 (Re J) and r0 + 1 (Im J)
#pragma unroll 4
            for (int k = 0; k < P::KP; ++k) {
                const float re = k < NJ ? J[k].re : 0.f, im = k < NJ ? J[k].im : 0.f;
                const float rh = tf32_hi(re), ih = tf32_hi(im);
                *reinterpret_cast<float *>(s.a_hi + core_offset(r0, k, P::KP)) = rh;
                *reinterpret_cast<float *>(s.a_lo + core_offset(r0, k, P::KP)) = re - rh;
                *reinterpret_cast<float *>(s.a_hi + core_offset(r0 + 1, k, P::KP)) = ih;
                *reinterpret_cast<float *>(s.a_lo + core_offset(r0 + 1, k, P::KP)) = im - ih;
            }
        }
        mma_round<NJ>(s);
        float m = 0.f;
        if (!s.failed) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t trow = *s.tmem_slot + ((uint32_t)((t >> 5) * 32) << 16);
#pragma unroll 1
            for (int c0 = 0; c0 < P::NP; c0 += 16) {
                float z[16];
                ld_cols<16>(trow + c0, z);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int c = c0 + i;
                    if (c < NJ) {
                        const uint32_t o = core_offset(t, c, P::KP);
                        const float a = *reinterpret_cast<const float *>(s.a_hi + o) +
                                        *reinterpret_cast<const float *>(s.a_lo + o);
                        m += a * z[i];
                    }
                }
            }
        }
        const float pair = m + __shfl_xor_sync(0xffffffffu, m, 1);
        if (!(t & 1)) s.out[64 * round + (t >> 1)] = pair;
        round_done();
    }
    return s.failed ? 0.f : s.out[t];
}

// One call: every thread of the block passes its (point, helicity) row's
// amplitudes J (NJ complex) and receives sum_kl Re(conj(J_k) C_kl J_l)
// (numerators only: divide by the colour denominator).  Must be called by
// all 128 threads.
template <int NJ>
MF_DEV float colour_sum(State &s, const cx<float> *J) {
    using P = Plan<NJ>;
    if constexpr (P::STACKED) {
        return colour_sum_stacked<NJ>(s, J);
    } else {
        const int r = threadIdx.x;
        if (!s.failed) {
            // this row of A_hi and A_lo: [Re J | Im J], zero padded to KP
#pragma unroll
            for (int k = 0; k < P::KP; ++k) {
                const float a = k < NJ ? J[k].re : (k < 2 * NJ ? J[k - NJ].im : 0.f);
                const float hi = tf32_hi(a);
                *reinterpret_cast<float *>(s.a_hi + core_offset(r, k, P::KP)) = hi;
                *reinterpret_cast<float *>(s.a_lo + core_offset(r, k, P::KP)) = a - hi;
            }
        }
        mma_round<NJ>(s);
        float m = 0.f;
        if (!s.failed) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // this row of Z, 16 columns at a time (warp w reads lanes 32w .. 32w+31)
            const uint32_t trow = *s.tmem_slot + ((uint32_t)((threadIdx.x >> 5) * 32) << 16);
#pragma unroll
            for (int c0 = 0; c0 < P::NP; c0 += 16) {
                float z[16];
                ld_cols<16>(trow + c0, z);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int c = c0 + i;
                    if (c < NJ) m += J[c].re * z[i];
                    else if (c < 2 * NJ) m += J[c - NJ].im * z[i];
                }
            }
        }
        round_done();
        return m;
    }
}

// Release the tensor memory (warp 0) once every MMA the block issued has
// completed: thread 0 commits them to the drain barrier (a commit tracks all
// earlier MMAs of the issuing thread) and every thread waits for its first
// phase with the full limit.  All threads.
template <int NJ>
MF_DEV void teardown(State &s) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x == 0)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(s.drain))
                     : "memory");
    if (!wait_phase(s.drain, 0u)) {
        s.failed = true;
        if (s.err) atomicExch(s.err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*s.tmem_slot), "r"(Plan<NJ>::COLS));
    }
}

}  // namespace tc
}  // namespace mf
