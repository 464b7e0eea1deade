// tbs_fft.cuh -- register-resident Stockham FFT engine for the Born-series
// passes (complex64, sm_103a).
//
// A line of length M (power of two, 16..4096) is held by T = M/E threads, E
// values each.  Thread t owns the "natural strided" elements t + T*m, m < E,
// in a[m] -- the order in which lines are loaded from and stored to global
// memory (coalesced: consecutive t touch consecutive addresses).
//
// Each stage of radix R (Stockham autosort, decimation in time; Govindaraju et
// al., SC'08) runs B = E/R butterflies per thread, j = t + q*T, on inputs
// x[j + r*M/R] (= slot a[q + r*B]), twiddled by w^{(j mod Ns) r M/(Ns R)} and
// transformed by an R-point DFT in registers; outputs go to positions
// (j div Ns) Ns R + (j mod Ns) + r Ns.  Between stages the outputs pass
// through shared memory; the last stage's outputs land exactly on the
// thread's natural strided slots, so a forward transform, a pointwise
// product and an inverse transform chain without any exchange in between.
//
// Shared memory positions are padded by one element every 16 (p + p/16),
// which keeps both the stride-R writes of the first stage and the unit-stride
// reads conflict-free for 8-byte elements.
//
// Twiddles come from a per-M table tw[k] = exp(-2 pi i k / M) built once in
// FP64 (sincospi) and rounded to float; the inverse uses conj.  Every
// butterfly is written as layers of two-point butterflies in FMA form
// (p + w q by two FMAs per component, p - w q = 2p - (p + w q) by one), with
// the stage twiddle W^r folded into those layers: a twiddled radix-16
// butterfly takes 192 FP32 instructions and eight table twiddles (no
// products of twiddles), against 256 for twiddle products followed by a
// plain 16-point DFT.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace tbs {

// compile-time loop: f(std::integral_constant<int, i>) for i in [0, N)
template <int N, class F, int... I>
__host__ __device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__host__ __device__ __forceinline__ void static_for(F &&f) {
    static_for_impl<N>(f, std::make_integer_sequence<int, N>{});
}

// ---- complex helpers -------------------------------------------------------
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// multiply by DIR * i  (DIR = -1: forward, +1: inverse)
template <int DIR>
__host__ __device__ __forceinline__ float2 mul_diri(float2 v) {
    return DIR > 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
}

// cos(2 pi e / 16), e in [0, 16)
__host__ __device__ constexpr float cos16(int e) {
    return e == 0 ? 1.0f : e == 1 ? 0.92387953251128674f : e == 2 ? 0.70710678118654752f
         : e == 3 ? 0.38268343236508978f : e == 4 ? 0.0f : e == 5 ? -0.38268343236508978f
         : e == 6 ? -0.70710678118654752f : e == 7 ? -0.92387953251128674f : e == 8 ? -1.0f
         : e == 9 ? -0.92387953251128674f : e == 10 ? -0.70710678118654752f
         : e == 11 ? -0.38268343236508978f : e == 12 ? 0.0f : e == 13 ? 0.38268343236508978f
         : e == 14 ? 0.70710678118654752f : 0.92387953251128674f;
}

// v * exp(DIR * 2 pi i e / 16)
template <int EXP, int DIR>
__device__ __forceinline__ float2 mul_w16(float2 v) {
    constexpr int e = ((EXP % 16) + 16) % 16;
    if constexpr (e == 0) {
        return v;
    } else if constexpr (e == 4) {
        return mul_diri<DIR>(v);
    } else if constexpr (e == 8) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (e == 12) {
        return mul_diri<-DIR>(v);
    } else {
        constexpr float c = cos16(e);
        constexpr float s = DIR * cos16((e + 12) % 16);  // sin(2 pi e/16) = cos(2 pi (e-4)/16)
        return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
    }
}

// ---- two-point butterflies ------------------------------------------------
// (p, q) <- (p + w q, p - w q) for a general w: six FP32 instructions.
__host__ __device__ __forceinline__ void bfly(float2 &p, float2 &q, float2 w) {
    const float sx = fmaf(w.x, q.x, fmaf(-w.y, q.y, p.x));
    const float sy = fmaf(w.x, q.y, fmaf(w.y, q.x, p.y));
    q = make_float2(fmaf(2.f, p.x, -sx), fmaf(2.f, p.y, -sy));
    p = make_float2(sx, sy);
}

// (p, q) <- (p + w q, p - w q) for w = exp(DIR 2 pi i e / 16), e a constant:
// w = 1, -1 and +-i take four additions, the others six FMA-form operations.
template <int EXP, int DIR>
__host__ __device__ __forceinline__ void bfly_c(float2 &p, float2 &q) {
    constexpr int e = ((EXP % 16) + 16) % 16;
    if constexpr (e == 0) {
        const float2 s = cadd(p, q);
        q = csub(p, q);
        p = s;
    } else if constexpr (e == 8) {
        const float2 s = csub(p, q);
        q = cadd(p, q);
        p = s;
    } else if constexpr (e == 4 || e == 12) {
        const float2 t = mul_diri<e == 4 ? DIR : -DIR>(q);
        const float2 s = cadd(p, t);
        q = csub(p, t);
        p = s;
    } else {
        constexpr float c = cos16(e);
        constexpr float sn = DIR * cos16((e + 12) % 16);  // DIR sin(2 pi e / 16)
        bfly(p, q, make_float2(c, sn));
    }
}

// a table twiddle (forward value t) in the direction of the transform
template <int DIR>
__host__ __device__ __forceinline__ float2 tw_dir(float2 t) { return DIR < 0 ? t : make_float2(t.x, -t.y); }

// ---- radix plans ----------------------------------------------------------
// RS = 0: M = 16^a * r (r in {1,2,4,8}); 512 uses three radix-8 stages.
// RS = 1: radix-8 stages, M = 8^a * r (r in {1,2,4}); 4096 = 8 x 8 x 8 x 8
// (one more exchange than 16 x 16 x 16, simpler butterflies).
template <int M, int RS = 0>
struct RadixPlan {
    __host__ __device__ static constexpr int log2m() { int l = 0, x = M; while (x > 1) { x >>= 1; l++; } return l; }
    __host__ __device__ static constexpr int n16() {
        return RS == 1 ? log2m() / 3 : M == 512 ? 0 : log2m() / 4;  // stages of the main radix
    }
    __host__ __device__ static constexpr int rem() {
        return RS == 1 ? (1 << (log2m() % 3)) : M == 512 ? 8 : (1 << (log2m() % 4));
    }
    static constexpr int MAIN = RS == 1 ? 8 : 16;
    static constexpr int NS = (RS == 0 && M == 512) ? 3 : n16() + (rem() > 1 ? 1 : 0);
    __host__ __device__ static constexpr int radix(int s) {
        return (RS == 0 && M == 512) ? 8 : (s < n16() ? MAIN : rem());
    }
    __host__ __device__ static constexpr int span(int s) {  // product of the radices before stage s
        int p = 1;
        for (int i = 0; i < s; i++) p *= radix(i);
        return p;
    }
    __host__ __device__ static constexpr int max_radix() {
        return (RS == 0 && M == 512) ? 8 : (n16() > 0 ? MAIN : rem());
    }
};

// Twiddles of one butterfly with stage twiddle W = tw[e] (forward values; the
// inverse conjugates them), every one a single table entry:
//   R = 2:  p[0] = W
//   R = 4:  u1 = W, u2 = W^2
//   R = 8:  u1 = W^2, u2 = W^4, p[k] = W w8^k (k < 2)
//   R = 16: u1 = W^4, u2 = W^8, p[k] = W w16^k (k < 4), q[k] = W^2 w8^k (k < 2)
// with w_n = exp(-2 pi i / n).  The set is shared by all lines a thread
// transforms at the same position, and by both directions.
template <int R>
struct TwSet {
    float2 u1, u2;
    float2 p[R == 16 ? 4 : R == 8 ? 2 : 1];
    float2 q[2];
};

template <int M, int R>
__device__ __forceinline__ TwSet<R> load_twiddles(const float2 *__restrict__ tw, int e) {
    TwSet<R> s;
    if constexpr (R == 2) {
        s.p[0] = __ldg(tw + e);
    } else if constexpr (R == 4) {
        s.u1 = __ldg(tw + e);
        s.u2 = __ldg(tw + 2 * e);
    } else if constexpr (R == 8) {
        s.u1 = __ldg(tw + 2 * e);
        s.u2 = __ldg(tw + 4 * e);
        s.p[0] = __ldg(tw + e);
        s.p[1] = __ldg(tw + e + M / 8);
    } else {
        s.u1 = __ldg(tw + 4 * e);
        s.u2 = __ldg(tw + 8 * e);
#pragma unroll
        for (int k = 0; k < 4; k++) s.p[k] = __ldg(tw + e + k * (M / 16));
        s.q[0] = __ldg(tw + 2 * e);
        s.q[1] = __ldg(tw + 2 * e + M / 8);
    }
    return s;
}

// ---- R-point butterflies: X[k] = sum_r x[r] W^r exp(DIR 2 pi i r k / R) ----
// TW = false: W = 1 (first stage).  ZIN: x[r] = 0 for r >= R/2 (zero-padded
// input; those registers are not read).  Outputs unneeded by the caller are
// removed by the compiler as dead code.
//
// Radix 4: the even and odd halves, X[k] = (x0 + W^2 (-1)^k x2) +
// W w4^k (x1 + W^2 (-1)^k x3), i.e. two butterflies with W^2, then two with
// W and W w4.
template <int DIR, bool TW, bool ZIN>
__host__ __device__ __forceinline__ void bf4(float2 &x0, float2 &x1, float2 &x2, float2 &x3, float2 u1, float2 u2) {
    if constexpr (ZIN) {
        static_assert(!TW, "zero-padded input only in a first stage");
        x2 = x0;
        x3 = x1;
    } else if constexpr (TW) {
        bfly(x0, x2, u2);
        bfly(x1, x3, u2);
    } else {
        bfly_c<0, DIR>(x0, x2);
        bfly_c<0, DIR>(x1, x3);
    }
    // (x0, x1) -> X0, X2;  (x2, x3) -> X1, X3
    if constexpr (TW) {
        bfly(x0, x1, u1);
        bfly(x2, x3, mul_diri<DIR>(u1));
    } else {
        bfly_c<0, DIR>(x0, x1);
        bfly_c<4, DIR>(x2, x3);
    }
    const float2 y1 = x2;
    x2 = x1;
    x1 = y1;
}

template <int R, int DIR, bool TW, bool ZIN>
__host__ __device__ __forceinline__ void butterfly(float2 (&v)[R], const TwSet<R> &s) {
    if constexpr (R == 2) {
        if constexpr (ZIN) {
            v[1] = v[0];
        } else if constexpr (TW) {
            bfly(v[0], v[1], tw_dir<DIR>(s.p[0]));
        } else {
            bfly_c<0, DIR>(v[0], v[1]);
        }
    } else if constexpr (R == 4) {
        bf4<DIR, TW, ZIN>(v[0], v[1], v[2], v[3], tw_dir<DIR>(s.u1), tw_dir<DIR>(s.u2));
    } else if constexpr (R == 8) {
        // x[n2 + 2 n1] -> X[k1 + 4 k2]: radix-4 over n1 with W^2 for each n2,
        // then radix-2 over n2 with W w8^k1
        const float2 u1 = tw_dir<DIR>(s.u1), u2 = tw_dir<DIR>(s.u2);
        float2 z[2][4];
#pragma unroll
        for (int n2 = 0; n2 < 2; n2++) {
            z[n2][0] = v[n2], z[n2][1] = v[n2 + 2], z[n2][2] = v[n2 + 4], z[n2][3] = v[n2 + 6];
            bf4<DIR, TW, ZIN>(z[n2][0], z[n2][1], z[n2][2], z[n2][3], u1, u2);
        }
        if constexpr (TW) {
            const float2 p0 = tw_dir<DIR>(s.p[0]), p1 = tw_dir<DIR>(s.p[1]);
            bfly(z[0][0], z[1][0], p0);
            bfly(z[0][1], z[1][1], p1);
            bfly(z[0][2], z[1][2], mul_diri<DIR>(p0));
            bfly(z[0][3], z[1][3], mul_diri<DIR>(p1));
        } else {
            bfly_c<0, DIR>(z[0][0], z[1][0]);
            bfly_c<2, DIR>(z[0][1], z[1][1]);
            bfly_c<4, DIR>(z[0][2], z[1][2]);
            bfly_c<6, DIR>(z[0][3], z[1][3]);
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; k1++) {
            v[k1] = z[0][k1];
            v[k1 + 4] = z[1][k1];
        }
    } else {
        static_assert(R == 16, "radix 2, 4, 8 or 16");
        // x[n2 + 4 n1] -> X[k1 + 4 k2]: radix-4 over n1 with W^4 for each
        // n2, then radix-4 over n2 with W w16^k1 (its square W^2 w8^k1)
        const float2 u1 = tw_dir<DIR>(s.u1), u2 = tw_dir<DIR>(s.u2);
        float2 z[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; n2++) {
            z[n2][0] = v[n2], z[n2][1] = v[n2 + 4], z[n2][2] = v[n2 + 8], z[n2][3] = v[n2 + 12];
            bf4<DIR, TW, ZIN>(z[n2][0], z[n2][1], z[n2][2], z[n2][3], u1, u2);
        }
        // z[n2][k1]; outer radix 4 over n2 for each k1
        auto outer = [&](auto kc) {
            constexpr int k1 = decltype(kc)::value;
            float2 b0 = z[0][k1], b1 = z[1][k1], b2 = z[2][k1], b3 = z[3][k1];
            if constexpr (TW) {
                const float2 q01 = tw_dir<DIR>(s.q[k1 & 1]);
                const float2 q = (k1 & 2) ? mul_diri<DIR>(q01) : q01;  // W^2 w8^k1
                const float2 p = tw_dir<DIR>(s.p[k1]);                // W w16^k1
                bfly(b0, b2, q);
                bfly(b1, b3, q);
                bfly(b0, b1, p);
                bfly(b2, b3, mul_diri<DIR>(p));
            } else {
                bfly_c<2 * k1, DIR>(b0, b2);
                bfly_c<2 * k1, DIR>(b1, b3);
                bfly_c<k1, DIR>(b0, b1);
                bfly_c<k1 + 4, DIR>(b2, b3);
            }
            // b0 = X[k1], b1 = X[k1 + 8], b2 = X[k1 + 4], b3 = X[k1 + 12]
            v[k1] = b0;
            v[k1 + 8] = b1;
            v[k1 + 4] = b2;
            v[k1 + 12] = b3;
        };
        static_for<4>(outer);
    }
}

// ---- asynchronous global -> shared copies (cp.async, completion per thread
// via commit/wait groups; no spin loops) -------------------------------------
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// padded shared-memory position
__device__ __forceinline__ int padpos(int p) { return p + (p >> 4); }
__host__ __device__ constexpr int padded_len(int m) { return m + (m >> 4); }

// Shared-memory view of the L lines a thread transforms: element p of line l
// sits at base[l * lstride + padpos(p)].  Lines are transformed and exchanged
// one after the other, so only one line's butterfly outputs are live at a
// time.  A line stride of 16 (mod 32) banks keeps two lines' accesses in one
// warp conflict-free.
// IL (two lines only): the lines are interleaved instead, element p of line
// l at base[2 padpos(p) + l], so that a thread moves both lines' element p
// with one 16-byte access (lstride unused).
template <int L, bool IL = false>
struct Lines {
    static_assert(!IL || L == 2, "interleaving pairs two lines");
    float2 *base;
    int lstride;
    __device__ __forceinline__ float2 ld(int l, int p) const {
        return IL ? base[2 * padpos(p) + l] : base[l * lstride + padpos(p)];
    }
    __device__ __forceinline__ void st(int l, int p, float2 v) const {
        if (IL)
            base[2 * padpos(p) + l] = v;
        else
            base[l * lstride + padpos(p)] = v;
    }
};

// All twiddles a thread t needs for one transform of length M: one set per
// stage S > 0 and per butterfly q.  They depend on t only, so a thread can
// load them once and reuse them for every line, for both directions and for
// every tile it processes.
template <int M, int E, int RS = 0>
struct ThreadTwiddles {
    using P = RadixPlan<M, RS>;
    static constexpr int B1 = P::NS > 1 ? E / P::radix(P::NS > 1 ? 1 : 0) : 1;
    static constexpr int B2 = P::NS > 2 ? E / P::radix(P::NS > 2 ? 2 : 0) : 1;
    static constexpr int B3 = P::NS > 3 ? E / P::radix(P::NS > 3 ? 3 : 0) : 1;
    TwSet<P::radix(P::NS > 1 ? 1 : 0)> s1[B1];
    TwSet<P::radix(P::NS > 2 ? 2 : 0)> s2[B2];
    TwSet<P::radix(P::NS > 3 ? 3 : 0)> s3[P::NS > 3 ? B3 : 1];

    __device__ __forceinline__ void load(const float2 *__restrict__ tw, int t) {
        constexpr int T = M / E;
        if constexpr (P::NS > 1) {
            constexpr int R = P::radix(1), Ns = P::span(1);
#pragma unroll
            for (int q = 0; q < B1; q++) s1[q] = load_twiddles<M, R>(tw, ((t + q * T) & (Ns - 1)) * (M / (Ns * R)));
        }
        if constexpr (P::NS > 2) {
            constexpr int R = P::radix(2), Ns = P::span(2);
#pragma unroll
            for (int q = 0; q < B2; q++) s2[q] = load_twiddles<M, R>(tw, ((t + q * T) & (Ns - 1)) * (M / (Ns * R)));
        }
        if constexpr (P::NS > 3) {
            constexpr int R = P::radix(3), Ns = P::span(3);
#pragma unroll
            for (int q = 0; q < B3; q++) s3[q] = load_twiddles<M, R>(tw, ((t + q * T) & (Ns - 1)) * (M / (Ns * R)));
        }
    }
    template <int S, int Q>
    __device__ __forceinline__ const auto &get() const {
        if constexpr (S == 1) return s1[Q];
        else if constexpr (S == 2) return s2[Q];
        else return s3[Q];
    }
};

// One stage S of the engine for direction DIR on L lines per thread.
// Barrier over the threads that share the exchange lines: the whole block,
// or (GroupSync) a named barrier over a warp-aligned group of `count` threads.
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct GroupSync {
    int id, count;
    __device__ __forceinline__ void operator()() const {
        asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
    }
};

// WAR: before storing, wait until every thread's reads of the line are done
// (false only where a barrier since the line's last read already ensures it).
// ZIN (stage 0 only): the upper half of every butterfly's inputs, slots
// a[m] with m >= E/2, is zero (zero-padded lines) and is not read.
template <int M, int E, int DIR, int S, int L, class TWS, class SYNC = BlockSync, bool WAR = true, bool ZIN = false,
          bool IL = false, int RS = 0>
__device__ __forceinline__ void fft_stage(float2 (&a)[L][E], const Lines<L, IL> &sm, int t,
                                          const float2 *__restrict__ tw, const TWS *twr,
                                          const SYNC &sync = SYNC()) {
    using P = RadixPlan<M, RS>;
    constexpr int R = P::radix(S);
    constexpr int Ns = P::span(S);
    constexpr int B = E / R;
    constexpr int T = M / E;
    constexpr bool LAST = (S == P::NS - 1);
    static_assert(E % R == 0, "radix must divide E");
    static_assert(!ZIN || S == 0, "zero-padded input only in the first stage");
    if constexpr (S > 0) {
        sync();  // previous stage's outputs are in shared memory
        if constexpr (T % 16 == 0 && IL) {
            // both lines' element at once; padpos(t + T s) = padpos(t) + s (T + T/16)
            const float4 *rp = reinterpret_cast<const float4 *>(sm.base) + padpos(t);
#pragma unroll
            for (int q = 0; q < B; q++)
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const float4 w = rp[(q + r * B) * (T + T / 16)];
                    a[0][q + r * B] = make_float2(w.x, w.y);
                    a[1][q + r * B] = make_float2(w.z, w.w);
                }
        } else if constexpr (T % 16 == 0) {
            // padpos(t + T s) = padpos(t) + s (T + T/16): one base address,
            // constant offsets
            const float2 *rp = sm.base + padpos(t);
#pragma unroll
            for (int l = 0; l < L; l++)
#pragma unroll
                for (int q = 0; q < B; q++)
#pragma unroll
                    for (int r = 0; r < R; r++) a[l][q + r * B] = rp[l * sm.lstride + (q + r * B) * (T + T / 16)];
        } else {
#pragma unroll
            for (int l = 0; l < L; l++)
#pragma unroll
                for (int q = 0; q < B; q++)
#pragma unroll
                    for (int r = 0; r < R; r++) a[l][q + r * B] = sm.ld(l, t + T * (q + r * B));
        }
    }
    if constexpr (!LAST && WAR) sync();  // every read of this buffer is done
    static_for<B>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const int j = t + q * T;
        TwSet<R> ts{};
        if constexpr (S > 0) {
            if constexpr (std::is_same<TWS, void>::value) ts = load_twiddles<M, R>(tw, (j & (Ns - 1)) * (M / (Ns * R)));
            else ts = twr->template get<S, q>();
        }
        const int base = (j / Ns) * Ns * R + (j & (Ns - 1));
        if constexpr (IL && !LAST && (Ns == 1 || Ns % 16 == 0)) {
            // both lines' butterflies, then one 16-byte store per output pair
            float2 v0[R], v1[R];
#pragma unroll
            for (int r = 0; r < R; r++) {
                v0[r] = a[0][q + r * B];
                v1[r] = a[1][q + r * B];
            }
            butterfly<R, DIR, (S > 0), ZIN>(v0, ts);
            butterfly<R, DIR, (S > 0), ZIN>(v1, ts);
            float4 *wp = reinterpret_cast<float4 *>(sm.base) + padpos(base);
            constexpr int STEP = Ns == 1 ? 1 : Ns + Ns / 16;
#pragma unroll
            for (int r = 0; r < R; r++) wp[r * STEP] = make_float4(v0[r].x, v0[r].y, v1[r].x, v1[r].y);
            return;
        }
#pragma unroll
        for (int l = 0; l < L; l++) {
            float2 v[R];
#pragma unroll
            for (int r = 0; r < R; r++) v[r] = a[l][q + r * B];
            butterfly<R, DIR, (S > 0), ZIN>(v, ts);
            if constexpr (LAST) {
#pragma unroll
                for (int r = 0; r < R; r++) a[l][q + r * B] = v[r];
            } else if constexpr (Ns == 1 || Ns % 16 == 0) {
                // padpos(base + r Ns) = padpos(base) + r (Ns + Ns/16): for Ns = 1
                // the R outputs share one padding block (base is a multiple of R,
                // R <= 16), for Ns % 16 == 0 each step spans whole blocks
                float2 *wp = sm.base + l * sm.lstride + padpos(base);
                constexpr int STEP = Ns == 1 ? 1 : Ns + Ns / 16;
#pragma unroll
                for (int r = 0; r < R; r++) wp[r * STEP] = v[r];
            } else {
#pragma unroll
                for (int r = 0; r < R; r++) sm.st(l, base + r * Ns, v[r]);
            }
        }
    });
}

// Full transform of L lines: a[l][m] holds element t + T m of line l on entry
// and on exit.  Unnormalised: X[k] = sum_n x[n] exp(DIR 2 pi i n k / M).
// twr: the thread's preloaded twiddles (ThreadTwiddles<M, E>), or nullptr of
// type const void* to read them from the table tw.
// FRESH: no thread has read the line since the caller's last barrier over
// these threads, so stage 0 may store without its write-after-read barrier.
// ZIN: slots a[l][m], m >= E/2 (elements t + T m >= M/2) are zero on entry.
template <int M, int E, int DIR, int L, class TWS = void, class SYNC = BlockSync, bool FRESH = false,
          bool ZIN = false, bool IL = false, int RS = 0>
__device__ __forceinline__ void fft_lines(float2 (&a)[L][E], const Lines<L, IL> &sm, int t,
                                          const float2 *__restrict__ tw, const TWS *twr = nullptr,
                                          const SYNC &sync = SYNC()) {
    using P = RadixPlan<M, RS>;
    static_assert(P::NS <= 4, "up to four stages");
    fft_stage<M, E, DIR, 0, L, TWS, SYNC, !FRESH, ZIN, IL, RS>(a, sm, t, tw, twr, sync);
    if constexpr (P::NS > 1)
        fft_stage<M, E, DIR, (P::NS > 1 ? 1 : 0), L, TWS, SYNC, true, false, IL, RS>(a, sm, t, tw, twr, sync);
    if constexpr (P::NS > 2)
        fft_stage<M, E, DIR, (P::NS > 2 ? 2 : 0), L, TWS, SYNC, true, false, IL, RS>(a, sm, t, tw, twr, sync);
    if constexpr (P::NS > 3)
        fft_stage<M, E, DIR, (P::NS > 3 ? 3 : 0), L, TWS, SYNC, true, false, IL, RS>(a, sm, t, tw, twr, sync);
}

// ---- two lines, staggered ------------------------------------------------
// The stage of fft_stage split into its three phases for ONE line whose
// exchange buffer is `line` (padded positions; T = M/E must be a multiple of
// 16): load the stage's inputs, run its butterflies (outputs kept in a[],
// output r of butterfly q in slot q + r B), store them for the next stage.
template <int M, int E, int S>
__device__ __forceinline__ void stage_load(float2 (&a)[E], const float2 *line, int t) {
    using P = RadixPlan<M>;
    constexpr int R = P::radix(S), B = E / R, T = M / E;
    static_assert(T % 16 == 0, "constant-offset addressing");
    const float2 *rp = line + padpos(t);
#pragma unroll
    for (int q = 0; q < B; q++)
#pragma unroll
        for (int r = 0; r < R; r++) a[q + r * B] = rp[(q + r * B) * (T + T / 16)];
}

template <int M, int E, int DIR, int S, bool ZIN, class TWS>
__device__ __forceinline__ void stage_compute(float2 (&a)[E], const TWS &twr) {
    using P = RadixPlan<M>;
    constexpr int R = P::radix(S), B = E / R;
    static_for<B>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        TwSet<R> ts{};
        if constexpr (S > 0) ts = twr.template get<S, q>();
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = a[q + r * B];
        butterfly<R, DIR, (S > 0), ZIN>(v, ts);
#pragma unroll
        for (int r = 0; r < R; r++) a[q + r * B] = v[r];
    });
}

template <int M, int E, int S>
__device__ __forceinline__ void stage_store(const float2 (&a)[E], float2 *line, int t) {
    using P = RadixPlan<M>;
    constexpr int R = P::radix(S), Ns = P::span(S), B = E / R, T = M / E;
    static_assert(Ns == 1 || Ns % 16 == 0, "constant-offset addressing");
    constexpr int STEP = Ns == 1 ? 1 : Ns + Ns / 16;
#pragma unroll
    for (int q = 0; q < B; q++) {
        const int j = t + q * T;
        float2 *wp = line + padpos((j / Ns) * Ns * R + (j & (Ns - 1)));
#pragma unroll
        for (int r = 0; r < R; r++) wp[r * STEP] = a[q + r * B];
    }
}

// Full transforms of two lines A and B (each with its own exchange buffer and
// its own barrier, syncA / syncB over the same threads), staggered so that
// one line's shared-memory traffic and barrier overlap the other line's
// butterflies: per stage, A's and B's loads are issued back to back, then
// A's butterflies run while B's loads land, and B's while A's outputs are
// stored.  Same arithmetic, hence bitwise the same results, as fft_lines on
// each line.  FRESH: no thread has read either buffer since the last barrier
// of its line, so the first stores need no write-after-read barrier.
template <int M, int E, int DIR, bool FRESH, bool ZIN, class TWS, class SYNC>
__device__ __forceinline__ void fft_pair(float2 (&a)[E], float2 (&b)[E], float2 *la, float2 *lb, int t,
                                         const TWS &twr, const SYNC &syncA, const SYNC &syncB) {
    using P = RadixPlan<M>;
    static_assert(P::NS >= 2, "at least two stages");
    stage_compute<M, E, DIR, 0, ZIN>(a, twr);
    if constexpr (!FRESH) syncA();
    stage_store<M, E, 0>(a, la, t);
    stage_compute<M, E, DIR, 0, ZIN>(b, twr);
    if constexpr (!FRESH) syncB();
    stage_store<M, E, 0>(b, lb, t);
    static_for<P::NS>([&](auto sc) {
        constexpr int S = decltype(sc)::value;
        if constexpr (S > 0) {
            constexpr bool LAST = S == P::NS - 1;
            syncA();  // A's previous outputs are stored
            stage_load<M, E, S>(a, la, t);
            syncB();
            stage_load<M, E, S>(b, lb, t);
            stage_compute<M, E, DIR, S, false>(a, twr);
            if constexpr (!LAST) {
                syncA();  // every read of A's buffer is done
                stage_store<M, E, S>(a, la, t);
            }
            stage_compute<M, E, DIR, S, false>(b, twr);
            if constexpr (!LAST) {
                syncB();
                stage_store<M, E, S>(b, lb, t);
            }
        }
    });
}

}  // namespace tbs
