// Shared-memory Stockham FFT for one line of N points held by a team of
// threads (FP32 float2, FP64 double2 or double-float dfc).
//
// A team of T = N/E threads (E = 8, 16 or 32) transforms one line; thread t holds the E values at
// positions t + m*T (m = 0..E-1) in registers, both on entry and on exit (the
// Stockham autosort keeps that distribution, so a forward transform, a pointwise
// multiply and an inverse transform chain with no extra data movement).
//
// Radix plan: the first stage is radix 16 (or N for N < 16), then radix-16
// stages, then one radix 2/4/8 stage for the remaining bits (with 8 values per
// thread: radix-8 stages and a radix 2/4 tail).  Between stages the
// line goes through the team's shared-memory buffer, padded by one element per
// 16 so that the stride-16 stores of the first stage are bank-conflict free.
//
// Stage s with radix R and span P (product of the radices before it) computes,
// for each butterfly i in [0, N/R):  k = i mod P,
//   u_r = x[i + r N/R] * W_{PR}^{r k},  y = DFT_R(u),  out[(i/P) P R + k + r P] = y_r.
// DIR = -1 is the forward transform exp(-2 pi i k x / N); DIR = +1 the inverse
// (unnormalised).  Twiddles come either from the global table
// tw[j] = exp(-2 pi i j / N) or from a per-block shared copy laid out [k][r]
// per stage (conflict-free for consecutive k).
#pragma once

#include <cooperative_groups.h>
#include <type_traits>

#include "common.cuh"

namespace scint {

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// cos(2 pi j / 16) for any integer j; sin(2 pi j/16) = cos(2 pi (j-4)/16)
__host__ __device__ constexpr double cos16(int j) {
    switch (((j % 16) + 16) % 16) {
        case 0: return 1.0;
        case 1: return 0.92387953251128675613;
        case 2: return 0.70710678118654752440;
        case 3: return 0.38268343236508977173;
        case 4: return 0.0;
        case 5: return -0.38268343236508977173;
        case 6: return -0.70710678118654752440;
        case 7: return -0.92387953251128675613;
        case 8: return -1.0;
        case 9: return -0.92387953251128675613;
        case 10: return -0.70710678118654752440;
        case 11: return -0.38268343236508977173;
        case 12: return 0.0;
        case 13: return 0.38268343236508977173;
        case 14: return 0.70710678118654752440;
        default: return 0.92387953251128675613;
    }
}

// a * exp(DIR * 2 pi i J16 / 16), J16 a compile-time multiple of 1/16 turn
template <int J16, int DIR, typename C>
SCINT_DEV C rot16(C a) {
    constexpr int j = ((J16 % 16) + 16) % 16;
    using Rl = typename real_of<C>::type;
    if constexpr (j == 0) {
        return a;
    } else if constexpr (j == 4) {
        return mul_i<DIR>(a);
    } else if constexpr (j == 8) {
        return make_c<C>(0, 0) - a;
    } else if constexpr (j == 12) {
        return mul_i<-DIR>(a);
    } else {
        constexpr Rl c = (Rl)cos16(j);
        constexpr Rl s = (Rl)(DIR * cos16(j - 4));
        if constexpr (std::is_same<C, dfc>::value) {
            return cmul(a, dfc{c, s});
        } else {
            C r;
            r.x = a.x * c - a.y * s;
            r.y = a.x * s + a.y * c;
            return r;
        }
    }
}

// ---- in-register DFTs, natural order in and out ---------------------------
template <int DIR, typename C>
SCINT_DEV void dft2(C& a, C& b) {
    const C t = a - b;
    a = a + b;
    b = t;
}

template <int DIR, typename C>
SCINT_DEV void dft4(C& a0, C& a1, C& a2, C& a3) {
    const C t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3;
    const C t3 = mul_i<DIR>(a1 - a3);
    a0 = t0 + t2;
    a2 = t0 - t2;
    a1 = t1 + t3;
    a3 = t1 - t3;
}

template <int R, int DIR, typename C>
SCINT_DEV void dft(C* x) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        dft2<DIR>(x[0], x[1]);
    } else if constexpr (R == 4) {
        dft4<DIR>(x[0], x[1], x[2], x[3]);
    } else if constexpr (R == 8) {
        // n = n1 + 2 n2, k = 4 k1 + k2
#pragma unroll
        for (int n1 = 0; n1 < 2; ++n1) dft4<DIR>(x[n1], x[n1 + 2], x[n1 + 4], x[n1 + 6]);
        x[3] = rot16<2, DIR>(x[3]);   // W8^1
        x[5] = rot16<4, DIR>(x[5]);   // W8^2
        x[7] = rot16<6, DIR>(x[7]);   // W8^3
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) dft2<DIR>(x[2 * k2], x[2 * k2 + 1]);
        C y[8];
#pragma unroll
        for (int k1 = 0; k1 < 2; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) y[4 * k1 + k2] = x[k1 + 2 * k2];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = y[i];
    } else if constexpr (R == 16) {
        // n = n1 + 4 n2, k = 4 k1 + k2
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) dft4<DIR>(x[n1], x[n1 + 4], x[n1 + 8], x[n1 + 12]);
        // a[n1][k2] sits at x[n1 + 4 k2]; multiply by W16^(n1 k2)
        x[5] = rot16<1, DIR>(x[5]);
        x[9] = rot16<2, DIR>(x[9]);
        x[13] = rot16<3, DIR>(x[13]);
        x[6] = rot16<2, DIR>(x[6]);
        x[10] = rot16<4, DIR>(x[10]);
        x[14] = rot16<6, DIR>(x[14]);
        x[7] = rot16<3, DIR>(x[7]);
        x[11] = rot16<6, DIR>(x[11]);
        x[15] = rot16<9, DIR>(x[15]);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) dft4<DIR>(x[4 * k2], x[4 * k2 + 1], x[4 * k2 + 2], x[4 * k2 + 3]);
        C y[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) y[4 * k1 + k2] = x[k1 + 4 * k2];
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = y[i];
    }
}

// ---- radix 16 in FP32 with the twiddle products fused into the butterflies ----
// A radix-4 butterfly whose second and fourth inputs carry a twiddle (a0 + a2 w2,
// a0 - a2 w2, ...) takes the product into the sum by FMAs: y + x w in four FMAs and
// the difference as 2 y - (y + x w) in two, where a product then a sum and a difference
// take eight.  In a radix-16 butterfly this applies to the external twiddles of the
// first layer (stages after the first) and to the internal W16 rotations of the second,
// 26 of its ~290 instructions.  The rounding differs from the plain form only in
// the order of the operations.
SCINT_DEV float2 cfma(float2 x, float2 w, float2 y) {     // y + x w
    return make_float2(fmaf(x.x, w.x, fmaf(-x.y, w.y, y.x)), fmaf(x.x, w.y, fmaf(x.y, w.x, y.y)));
}
SCINT_DEV float2 twice_minus(float2 a, float2 b) {       // 2 a - b
    return make_float2(fmaf(2.0f, a.x, -b.x), fmaf(2.0f, a.y, -b.y));
}
// the factor rot16<J16, DIR> multiplies by, as a complex number
template <int J16, int DIR> SCINT_DEV float2 rot16_w() {
    return make_float2((float)cos16(J16), (float)(DIR * cos16(J16 - 4)));
}
// external twiddle of the stage: x W^rk for the forward transform, x conj(W^rk) for the inverse
template <int DIR> SCINT_DEV float2 tw_w(float2 w) { return DIR < 0 ? w : conjc(w); }

// the radix-16 butterfly of dft<16, DIR> on x[r] w[r] (w[0] = 1; TW = false: no external twiddles)
template <int DIR, bool TW>
SCINT_DEV void dft16_fused(float2* x, const float2* w) {
    // first layer over n2 for each n1 (n = n1 + 4 n2): inputs x[n1 + 4 n2] (times w[n1 + 4 n2])
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
        float2 t0, t1, t2, d;
        if constexpr (TW) {
            const float2 a0 = n1 == 0 ? x[0] : cmul(x[n1], tw_w<DIR>(w[n1]));
            const float2 a1 = cmul(x[n1 + 4], tw_w<DIR>(w[n1 + 4]));
            t0 = cfma(x[n1 + 8], tw_w<DIR>(w[n1 + 8]), a0);
            t1 = twice_minus(a0, t0);
            t2 = cfma(x[n1 + 12], tw_w<DIR>(w[n1 + 12]), a1);
            d = twice_minus(a1, t2);
        } else {
            t0 = x[n1] + x[n1 + 8];
            t1 = x[n1] - x[n1 + 8];
            t2 = x[n1 + 4] + x[n1 + 12];
            d = x[n1 + 4] - x[n1 + 12];
        }
        const float2 t3 = mul_i<DIR>(d);
        x[n1] = t0 + t2;
        x[n1 + 8] = t0 - t2;
        x[n1 + 4] = t1 + t3;
        x[n1 + 12] = t1 - t3;
    }
    // second layer over n1 for each k2: inputs x[4 k2 + n1] W16^(n1 k2)
    {   // k2 = 0: no rotation
        const float2 t0 = x[0] + x[2], t1 = x[0] - x[2], t2 = x[1] + x[3];
        const float2 t3 = mul_i<DIR>(x[1] - x[3]);
        x[0] = t0 + t2; x[2] = t0 - t2; x[1] = t1 + t3; x[3] = t1 - t3;
    }
    {   // k2 = 1: W^1, W^2, W^3
        const float2 t0 = cfma(x[6], rot16_w<2, DIR>(), x[4]);
        const float2 t1 = twice_minus(x[4], t0);
        const float2 a1 = rot16<1, DIR>(x[5]);
        const float2 t2 = cfma(x[7], rot16_w<3, DIR>(), a1);
        const float2 t3 = mul_i<DIR>(twice_minus(a1, t2));
        x[4] = t0 + t2; x[6] = t0 - t2; x[5] = t1 + t3; x[7] = t1 - t3;
    }
    {   // k2 = 2: W^2, W^4 (a quarter turn), W^6
        const float2 b2 = rot16<4, DIR>(x[10]);
        const float2 t0 = x[8] + b2, t1 = x[8] - b2;
        const float2 a1 = rot16<2, DIR>(x[9]);
        const float2 t2 = cfma(x[11], rot16_w<6, DIR>(), a1);
        const float2 t3 = mul_i<DIR>(twice_minus(a1, t2));
        x[8] = t0 + t2; x[10] = t0 - t2; x[9] = t1 + t3; x[11] = t1 - t3;
    }
    {   // k2 = 3: W^3, W^6, W^9
        const float2 t0 = cfma(x[14], rot16_w<6, DIR>(), x[12]);
        const float2 t1 = twice_minus(x[12], t0);
        const float2 a1 = rot16<3, DIR>(x[13]);
        const float2 t2 = cfma(x[15], rot16_w<9, DIR>(), a1);
        const float2 t3 = mul_i<DIR>(twice_minus(a1, t2));
        x[12] = t0 + t2; x[14] = t0 - t2; x[13] = t1 + t3; x[15] = t1 - t3;
    }
    float2 y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) y[4 * k1 + k2] = x[k1 + 4 * k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = y[i];
}

// ---- plan ----------------------------------------------------------------
// EPT = values held per thread (8, 16 or 32); each stage's butterflies are spread
// over the T = N/E threads of the line, E/R butterflies per thread.  The stages
// are radix 16 (EPT 16 or 32) or radix 8 (EPT 8), then one smaller tail stage.
// With EPT 8 every stage after the first must have N/R >= 16 (the padded
// addressing of the loads below), i.e. N >= 128.
template <int N, int EPT = 16>
struct FftPlan {
    static_assert(N >= 2 && (N & (N - 1)) == 0, "N must be a power of two");
    static_assert(EPT == 8 || EPT == 16 || EPT == 32, "8, 16 or 32 values per thread");
    static constexpr int LOG2N = ilog2(N);
    static constexpr int E = N < EPT ? N : EPT;          // values per thread
    static constexpr int T = N / E;                      // threads per line
    static constexpr int RB = EPT == 8 ? 8 : 16;         // radix of the full stages
    static constexpr int LB = ilog2(RB);
    static constexpr int R0 = N < RB ? N : RB;           // radix of the first stage
    static constexpr int REST = LOG2N - ilog2(R0);
    static constexpr int N16 = REST / LB;                // full stages after the first
    static constexpr int TAIL = REST % LB;               // bits of the last small stage
    static constexpr int NSTAGE = 1 + N16 + (TAIL ? 1 : 0);
    static constexpr int BUF = N + N / 16;               // padded buffer length
    __host__ __device__ static constexpr int radix(int s) { return s == 0 ? R0 : (s <= N16 ? RB : (1 << TAIL)); }
    __host__ __device__ static constexpr int span(int s) { return s == 0 ? 1 : span(s - 1) * radix(s - 1); }
    // shared twiddle table: for each stage s >= 1, entries [k][r - 1] = W_{PR}^{r k}
    __host__ __device__ static constexpr int twoff(int s) {
        return s <= 1 ? 0 : twoff(s - 1) + (radix(s - 1) - 1) * span(s - 1);
    }
    static constexpr int TWS = twoff(NSTAGE);            // table entries
};

// Fill a block's shared twiddle table from the global table tw[j * stride] = exp(-2 pi i j / N)
// (stride 2: the table of a line twice as long).
template <typename C, int N, int EPT = 16>
SCINT_DEV void fill_twiddle_table(C* tws, const C* __restrict__ tw, int tid, int nthreads, int stride = 1) {
    using Pl = FftPlan<N, EPT>;
#pragma unroll
    for (int s = 1; s < Pl::NSTAGE; ++s) {
        const int R = Pl::radix(s), P = Pl::span(s), base = Pl::twoff(s);
        for (int e = tid; e < (R - 1) * P; e += nthreads) {
            const int k = e / (R - 1), r = e % (R - 1) + 1;
            tws[base + e] = __ldg(tw + r * k * (N / (P * R)) * stride);
        }
    }
}

SCINT_DEV int pad16(int a) { return a + (a >> 4); }

template <typename C>
SCINT_DEV C ld_tw(const C* __restrict__ p) { return __ldg(p); }
template <>
SCINT_DEV dfc ld_tw<dfc>(const dfc* __restrict__ p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return dfc{dfl(v.x, v.y), dfl(v.z, v.w)};
}


// LW: lane width of the buffer.  Element e of the line sits at buf[pad16(e) * LW]
// (the caller offsets buf by its lane), so LW lines can share one interleaved
// buffer with consecutive threads of different lines hitting consecutive banks.
// Per-thread twiddle bases kept in registers across many transforms: for every
// stage s >= 1 and butterfly b of thread t, W^k and W^{4k} (W = W_{PR},
// k = (t + b T) mod P); the other powers are products of depth <= 3.
template <typename C, int N, int EPT>
struct TwiddleRegs {
    using Pl = FftPlan<N, EPT>;
    static constexpr int NS = Pl::NSTAGE > 1 ? Pl::NSTAGE : 2;
    static constexpr int MAXNB = Pl::E;     // >= E / R for every stage
    C w[NS][MAXNB][2];
    // tw[j * stride] = exp(-2 pi i j / N)
    SCINT_DEV void load(const C* __restrict__ tw, int t, int stride = 1) {
#pragma unroll
        for (int s = 1; s < Pl::NSTAGE; ++s) {
            const int R = Pl::radix(s), P = Pl::span(s);
#pragma unroll
            for (int b = 0; b < Pl::E / R; ++b) {
                const int k = (t + b * Pl::T) & (P - 1);
                const int step = k * (N / (P * R)) * stride;
                w[s][b][0] = __ldg(tw + step);
                w[s][b][1] = R >= 8 ? __ldg(tw + 4 * step) : w[s][b][0];
            }
        }
    }
};

// powers r = 1..R-1 of a base twiddle from (W^k, W^{4k})
template <int R, typename C>
SCINT_DEV void twiddle_powers(C w1, C w4, C (&w)[R]) {
    if constexpr (R >= 2) w[1] = w1;
    if constexpr (R >= 4) { w[2] = cmul(w1, w1); w[3] = cmul(w1, w[2]); }
    if constexpr (R >= 8) {
        w[4] = w4;
        w[5] = cmul(w4, w1);
        w[6] = cmul(w4, w[2]);
        w[7] = cmul(w4, w[3]);
    }
    if constexpr (R >= 16) {
        w[8] = cmul(w4, w4);
#pragma unroll
        for (int r = 9; r < 12; ++r) w[r] = cmul(w[8], w[r - 8]);
        w[12] = cmul(w[8], w4);
#pragma unroll
        for (int r = 13; r < 16; ++r) w[r] = cmul(w[12], w[r - 12]);
    }
}

// Twiddle source TWM: 0 = global table tw[j] = exp(-2 pi i j / N); 1 = the
// block's shared table (fill_twiddle_table; tw points to it); 2 = register
// bases (tr).
// CS = 1: the whole line sits in this block's shared buffer.  CS = 2: the line
// is split over a cluster of two blocks; elements [0, N/2) live in rank 0's
// buffer and [N/2, N) in rank 1's, each padded by pad16 of the local index, at
// the same offset in both blocks; t is the thread's index in the line's team
// across the cluster, and the stage barriers are cluster barriers.
// SUB: the threads that share the line buffers and synchronise: the whole block (0), or
// the SUB-thread part of the block that thread threadIdx.x belongs to, through the named
// barrier 1 + threadIdx.x / SUB (SUB a multiple of 32 dividing the block; barrier 0 stays
// the block's own) -- so that two independent teams can share one block.
template <int SUB> SCINT_DEV void team_sync() {
    if constexpr (SUB == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)threadIdx.x / SUB), "n"(SUB) : "memory");
}
template <int CS, int SUB = 0> SCINT_DEV void line_sync() {
    if constexpr (CS == 1) team_sync<SUB>();
    else cooperative_groups::this_cluster().sync();
}

// the two halves of a cluster barrier, for work between them
SCINT_DEV void cluster_arrive() { asm volatile("barrier.cluster.arrive.aligned;" ::: "memory"); }
SCINT_DEV void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }

// 32-bit shared::cluster address of the same shared-memory offset in block `rank`
// of the cluster (32-bit arithmetic instead of 64-bit generic pointers)
SCINT_DEV unsigned cluster_addr(const void* local, unsigned rank) {
    unsigned r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((unsigned)__cvta_generic_to_shared(local)), "r"(rank));
    return r;
}
template <typename C> SCINT_DEV C ld_cluster(unsigned addr);
template <>
SCINT_DEV float2 ld_cluster<float2>(unsigned addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
template <>
SCINT_DEV long long ld_cluster<long long>(unsigned addr) {
    long long v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}
template <>
SCINT_DEV double2 ld_cluster<double2>(unsigned addr) {
    double2 v;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(addr) : "memory");
    return v;
}
template <>
SCINT_DEV dfc ld_cluster<dfc>(unsigned addr) {
    float a, b, c, d;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(a), "=f"(b), "=f"(c), "=f"(d) : "r"(addr) : "memory");
    return dfc{dfl(a, b), dfl(c, d)};
}

// PP (ping-pong, CS = 1 only): stage s writes buffer s mod 2 (buf, buf1) and stage s + 1
// reads it, so a stage's reads and the next stage's writes touch different buffers
// and one barrier per stage suffices (in place: two).  The last stage reads buffer
// NSTAGE - 2; when that is buf, the next transform's first stage would overwrite it,
// so that case keeps a barrier after the reads.
template <typename C, int N, int DIR, int EPT, int LW, int TWM, int CS, int S, int TS = 1, bool PP = false, int SUB = 0>
SCINT_DEV void fft_stage(C (&v)[FftPlan<N, EPT>::E], C* buf, int t, const C* __restrict__ tw,
                         const TwiddleRegs<C, N, EPT>* tr, C* buf1 = nullptr) {
    using Pl = FftPlan<N, EPT>;
    constexpr int E = Pl::E, T = Pl::T;
    constexpr int R = Pl::radix(S), P = Pl::span(S), NB = E / R;
    constexpr bool FIRST = (S == 0), LAST = (S == Pl::NSTAGE - 1);
    constexpr int HALF = N / 2;
    static_assert(!PP || CS == 1, "ping-pong buffers are for unsplit lines");
    C* const rbuf = PP && (S % 2 == 0) ? buf1 : buf;    // written by stage S - 1
    C* const wbuf = PP && (S % 2 == 1) ? buf1 : buf;    // written by stage S
    C u[E];
    if constexpr (FIRST) {
        // butterfly b takes positions t + b T + r N/R = t + (b + r NB) T
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int r = 0; r < R; ++r) u[b * R + r] = v[b + r * NB];
    } else if constexpr (CS == 1) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            // N/R is a multiple of 16 here, so pad16(i + r N/R) = pad16(i) + r (N/R)(17/16).
#pragma unroll
            for (int r = 0; r < R; ++r) u[b * R + r] = rbuf[pad16(t + b * T) * LW + r * ((N / R) + (N / R) / 16) * LW];
        }
        if constexpr (!PP || (LAST && (Pl::NSTAGE - 2) % 2 == 0)) team_sync<SUB>();
    } else {
        // Split line: i < N/R <= N/2, so element i + r N/R is in the upper half
        // (rank 1's buffer, local index i + (r - R/2) N/R) iff r >= R/2.
        const unsigned cb0 = cluster_addr(buf, 0), cb1 = cluster_addr(buf, 1);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const unsigned off = (unsigned)(pad16(t + b * T) * LW * sizeof(C));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int rr = r < R / 2 ? r : r - R / 2;
                u[b * R + r] = ld_cluster<C>((r < R / 2 ? cb0 : cb1) + off +
                                             (unsigned)(rr * ((N / R) + (N / R) / 16) * LW * sizeof(C)));
            }
        }
        line_sync<CS, SUB>();
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int i = t + b * T;
        if constexpr (std::is_same<C, float2>::value && R == 16) {
            C w[R];
            if constexpr (!FIRST) {
                const int k = i & (P - 1);
                if constexpr (TWM == 2) {
                    twiddle_powers<R>(tr->w[S][b][0], tr->w[S][b][1], w);
                } else {
#pragma unroll
                    for (int r = 1; r < R; ++r)
                        w[r] = TWM == 1 ? tw[Pl::twoff(S) + k * (R - 1) + (r - 1)] : ld_tw(tw + r * k * (N / (P * R)) * TS);
                }
            }
            dft16_fused<DIR, !FIRST>(&u[b * R], w);
            continue;
        }
        if constexpr (!FIRST) {
            const int k = i & (P - 1);
            if constexpr (TWM == 2) {
                C w[R];
                twiddle_powers<R>(tr->w[S][b][0], tr->w[S][b][1], w);
#pragma unroll
                for (int r = 1; r < R; ++r) u[b * R + r] = DIR < 0 ? cmul(u[b * R + r], w[r]) : cmulc(u[b * R + r], w[r]);
            } else {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    // W_{PR}^{r k}: shared entry [k][r - 1] or global tw[r k N / (P R)]
                    const C w = TWM == 1 ? tw[Pl::twoff(S) + k * (R - 1) + (r - 1)]
                                         : ld_tw(tw + r * k * (N / (P * R)) * TS);
                    u[b * R + r] = DIR < 0 ? cmul(u[b * R + r], w) : cmulc(u[b * R + r], w);
                }
            }
        }
        dft<R, DIR>(&u[b * R]);
    }
    if constexpr (LAST) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int r = 0; r < R; ++r) v[b + r * NB] = u[b * R + r];
    } else {
        // Split line: with one butterfly per thread (NB = 1) and P <= T/2, the outputs
        // j + r P, j = (i/P) P R + i mod P, of thread i all lie in [0, N/2) iff i < T/2,
        // i.e. in the half its own block holds: every store is local, at j mod N/2.
        static_assert(CS == 1 || (NB == 1 && P <= T / 2), "split-line stores must stay in the block");
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int i = t + b * T;
            const int k = i & (P - 1);
            int j = (i - k) * R + k;
            if constexpr (CS == 2) j &= HALF - 1;
            // P >= 16: pad16(j + r P) = pad16(j) + r P (17/16); P == 1: j = i R and r < R <= 16
            // (j a multiple of R, so j + r stays in one group of 16); otherwise pad16 itself
            C* dst = wbuf + pad16(j) * LW;
#pragma unroll
            for (int r = 0; r < R; ++r)
                dst[(P >= 16 ? r * (P + P / 16) : (P == 1 ? r : pad16(j + r * P) - pad16(j))) * LW] = u[b * R + r];
        }
        line_sync<CS, SUB>();
        fft_stage<C, N, DIR, EPT, LW, TWM, CS, S + 1, TS, PP, SUB>(v, buf, t, tw, tr, buf1);
    }
}

// Transform the team's line in place (registers v, distribution t + m*T).
// Every thread of the block (of the cluster, for CS = 2) must call this the
// same number of times.
// TS: stride of the global table (TWM = 0), tw[j TS] = exp(-2 pi i j / N).
template <typename C, int N, int DIR, int EPT = 16, int LW = 1, int TWM = 0, int CS = 1, int TS = 1, int SUB = 0>
SCINT_DEV void fft_line(C (&v)[FftPlan<N, EPT>::E], C* buf, int t, const C* __restrict__ tw) {
    static_assert(TWM != 2, "register twiddles: use fft_line_tr");
    static_assert(CS == 1 || (CS == 2 && FftPlan<N, EPT>::NSTAGE > 1 && N >= 512), "split lines need N >= 512");
    fft_stage<C, N, DIR, EPT, LW, TWM, CS, 0, TS, false, SUB>(v, buf, t, tw, nullptr);
}

template <typename C, int N, int DIR, int EPT = 16, int LW = 1, int CS = 1, int SUB = 0>
SCINT_DEV void fft_line_tr(C (&v)[FftPlan<N, EPT>::E], C* buf, int t, const TwiddleRegs<C, N, EPT>& tr) {
    static_assert(CS == 1 || (CS == 2 && FftPlan<N, EPT>::NSTAGE > 1 && N >= 512), "split lines need N >= 512");
    fft_stage<C, N, DIR, EPT, LW, 2, CS, 0, 1, false, SUB>(v, buf, t, nullptr, &tr);
}

// Ping-pong forms (unsplit lines): buf1 is a second buffer laid out like buf.  Between
// two ping-pong transforms of the same buffers no barrier is needed; any other write
// to either buffer after one needs a __syncthreads first.
template <typename C, int N, int DIR, int EPT = 16, int LW = 1, int TWM = 0, int SUB = 0>
SCINT_DEV void fft_line_pp(C (&v)[FftPlan<N, EPT>::E], C* buf, C* buf1, int t, const C* __restrict__ tw) {
    static_assert(TWM != 2, "register twiddles: use fft_line_tr_pp");
    fft_stage<C, N, DIR, EPT, LW, TWM, 1, 0, 1, true, SUB>(v, buf, t, tw, nullptr, buf1);
}
template <typename C, int N, int DIR, int EPT = 16, int LW = 1, int SUB = 0>
SCINT_DEV void fft_line_tr_pp(C (&v)[FftPlan<N, EPT>::E], C* buf, C* buf1, int t, const TwiddleRegs<C, N, EPT>& tr) {
    fft_stage<C, N, DIR, EPT, LW, 2, 1, 0, 1, true, SUB>(v, buf, t, nullptr, &tr, buf1);
}

// ---- lines split by one radix-2 step over a two-block cluster ------------------
// Block r of the cluster holds the parity-r half-problem of an N-point line as a
// whole N/2 = H2-point line in its own shared memory.  After the inverse
// transforms of the halves (A' in block 0, B' in block 1, at n = t + m T), the
// decimation-in-time step y_n = A'_n + W^{-n} B'_n, y_{n+H2} = A'_n - W^{-n} B'_n
// (W = exp(-2 pi i / N), tw[j] = W^j) needs the other block's half: each block
// publishes its values in its buffer and fetches, for its quarter of the outputs
// (block 0: n < H2/2, block 1: n >= H2/2), the partner's.  emit(j, n, y_n, y_{n+H2})
// for n = t + (j + r E/2) T, j < E/2.  Ends with a cluster arrive: the caller
// waits (cluster_wait) before it next writes buf.
template <typename C, int H2, typename Emit>
SCINT_DEV void split_combine(C (&v)[FftPlan<H2>::E], C* buf, int t, int r, const C* __restrict__ tw, Emit&& emit) {
    using Pl = FftPlan<H2>;
    constexpr int T = Pl::T, E = Pl::E;
    static_assert(T % 16 == 0, "pad16(t + j T) = pad16(t) + j T 17/16");
#pragma unroll
    for (int m = 0; m < E; ++m) buf[pad16(t + m * T)] = v[m];
    line_sync<2>();
    const unsigned pb = cluster_addr(buf, (unsigned)(r ^ 1)) + (unsigned)(pad16(t + r * (E / 2) * T) * sizeof(C));
    C q[E / 2];
#pragma unroll
    for (int j = 0; j < E / 2; ++j) q[j] = ld_cluster<C>(pb + (unsigned)(j * (T + T / 16) * sizeof(C)));
    cluster_arrive();    // done with the partner's buffer
#pragma unroll
    for (int j = 0; j < E / 2; ++j) {
        const int n = t + (j + r * (E / 2)) * T;
        const C own = r == 0 ? v[j] : v[j + E / 2];
        const C A = r == 0 ? own : q[j], B = r == 0 ? q[j] : own;
        const C bw = cmulc(B, ld_tw(tw + n));
        emit(j, n, A + bw, A - bw);
    }
}

// Decimation in frequency for the forward transform: the parity-r half-problem's
// input, a_n = x_n + x_{n+H2} (r = 0) or b_n = (x_n - x_{n+H2}) W^n (r = 1).
template <typename C>
SCINT_DEV C split_dif(C x0, C x1, int r, int n, const C* __restrict__ tw) {
    return r == 0 ? x0 + x1 : cmul(x0 - x1, ld_tw(tw + n));
}

}  // namespace scint
