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
// FP64 (sincospi) and rounded to float; the inverse uses conj.  A radix-16
// butterfly loads six of its fifteen twiddles and forms the rest as products.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace tbs {

// compile-time loop: f(std::integral_constant<int, i>) for i in [0, N)
template <int N, class F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F &&f) {
    static_for_impl<N>(f, std::make_integer_sequence<int, N>{});
}

// ---- complex helpers -------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
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
__device__ __forceinline__ float2 mul_diri(float2 v) {
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

// ---- small DFTs in registers: X[k] = sum_n x[n] exp(DIR 2 pi i n k / R) ---
template <int DIR>
__device__ __forceinline__ void dft2(float2 &a, float2 &b) {
    float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
    float2 t0 = cadd(x0, x2), t1 = csub(x0, x2);
    float2 t2 = cadd(x1, x3), t3 = mul_diri<DIR>(csub(x1, x3));
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

template <int R, int DIR>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
    if constexpr (R == 2) {
        dft2<DIR>(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4<DIR>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        // 8 = 2 x 4: inputs x[4 n1 + n2]; inner 2-point DFTs over n1, twiddle
        // w8^{n2 k1}, outer 4-point DFTs over n2; output X[k1 + 2 k2].
        dft2<DIR>(v[0], v[4]);
        dft2<DIR>(v[1], v[5]);
        dft2<DIR>(v[2], v[6]);
        dft2<DIR>(v[3], v[7]);
        v[5] = mul_w16<2, DIR>(v[5]);
        v[6] = mul_w16<4, DIR>(v[6]);
        v[7] = mul_w16<6, DIR>(v[7]);
        dft4<DIR>(v[0], v[1], v[2], v[3]);
        dft4<DIR>(v[4], v[5], v[6], v[7]);
        // y[k1][k2] at v[4 k1 + k2] -> X[k1 + 2 k2]
        float2 o[8];
#pragma unroll
        for (int k1 = 0; k1 < 2; k1++)
#pragma unroll
            for (int k2 = 0; k2 < 4; k2++) o[k1 + 2 * k2] = v[4 * k1 + k2];
#pragma unroll
        for (int i = 0; i < 8; i++) v[i] = o[i];
    } else if constexpr (R == 16) {
        // 16 = 4 x 4: inputs x[4 n1 + n2]; inner 4-point DFTs over n1,
        // twiddle w16^{n2 k1}, outer 4-point DFTs over n2; X[k1 + 4 k2].
        dft4<DIR>(v[0], v[4], v[8], v[12]);
        dft4<DIR>(v[1], v[5], v[9], v[13]);
        dft4<DIR>(v[2], v[6], v[10], v[14]);
        dft4<DIR>(v[3], v[7], v[11], v[15]);
        // now v[4 k1 + n2] = y[n2][k1]
        v[5] = mul_w16<1, DIR>(v[5]);
        v[6] = mul_w16<2, DIR>(v[6]);
        v[7] = mul_w16<3, DIR>(v[7]);
        v[9] = mul_w16<2, DIR>(v[9]);
        v[10] = mul_w16<4, DIR>(v[10]);
        v[11] = mul_w16<6, DIR>(v[11]);
        v[13] = mul_w16<3, DIR>(v[13]);
        v[14] = mul_w16<6, DIR>(v[14]);
        v[15] = mul_w16<9, DIR>(v[15]);
        dft4<DIR>(v[0], v[1], v[2], v[3]);
        dft4<DIR>(v[4], v[5], v[6], v[7]);
        dft4<DIR>(v[8], v[9], v[10], v[11]);
        dft4<DIR>(v[12], v[13], v[14], v[15]);
        // v[4 k1 + k2] = X[k1 + 4 k2]: transpose 4 x 4
        float2 o[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; k1++)
#pragma unroll
            for (int k2 = 0; k2 < 4; k2++) o[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
        for (int i = 0; i < 16; i++) v[i] = o[i];
    }
}

// ---- radix plans ----------------------------------------------------------
// M = 16^a * r (r in {1,2,4,8}); 512 uses three radix-8 stages.
template <int M>
struct RadixPlan {
    __host__ __device__ static constexpr int log2m() { int l = 0, x = M; while (x > 1) { x >>= 1; l++; } return l; }
    __host__ __device__ static constexpr int n16() { return M == 512 ? 0 : log2m() / 4; }
    __host__ __device__ static constexpr int rem() { return M == 512 ? 8 : (1 << (log2m() % 4)); }
    static constexpr int NS = M == 512 ? 3 : n16() + (rem() > 1 ? 1 : 0);
    __host__ __device__ static constexpr int radix(int s) { return M == 512 ? 8 : (s < n16() ? 16 : rem()); }
    __host__ __device__ static constexpr int span(int s) {  // product of the radices before stage s
        int p = 1;
        for (int i = 0; i < s; i++) p *= radix(i);
        return p;
    }
    __host__ __device__ static constexpr int max_radix() { return M == 512 ? 8 : (n16() > 0 ? 16 : rem()); }
};

// Twiddles of one butterfly: v[r] *= W^r, W = tw[base] (conjugated for the
// inverse).  Only W^1..W^4 and, for R = 16, W^8 and W^12 are loaded; every
// other power is one product of two loaded values, so no twiddle carries more
// than one extra rounding.  The loaded set is shared by all lines a thread
// transforms at the same position.
template <int R>
struct TwSet {
    float2 w1, w2, w3, w4, w8, w12;
};

// Loads the forward-direction set; the inverse applies the conjugates.
template <int R>
__device__ __forceinline__ TwSet<R> load_twiddles(const float2 *__restrict__ tw, int base) {
    TwSet<R> s;
    s.w1 = __ldg(tw + base);
    if constexpr (R >= 4) {
        s.w2 = __ldg(tw + 2 * base);
        s.w3 = __ldg(tw + 3 * base);
    }
    if constexpr (R >= 8) s.w4 = __ldg(tw + 4 * base);
    if constexpr (R >= 16) {
        s.w8 = __ldg(tw + 8 * base);
        s.w12 = __ldg(tw + 12 * base);
    }
    return s;
}

// v[r] *= W^r (DIR < 0) or conj(W)^r (DIR > 0)
template <int R, int DIR>
__device__ __forceinline__ void apply_twiddles(float2 (&v)[R], const TwSet<R> &s) {
    auto mul = [](float2 x, float2 w) { return DIR < 0 ? cmul(x, w) : cmulc(x, w); };
    v[1] = mul(v[1], s.w1);
    if constexpr (R >= 4) {
        v[2] = mul(v[2], s.w2);
        v[3] = mul(v[3], s.w3);
    }
    if constexpr (R >= 8) {
        v[4] = mul(v[4], s.w4);
        v[5] = mul(v[5], cmul(s.w4, s.w1));
        v[6] = mul(v[6], cmul(s.w4, s.w2));
        v[7] = mul(v[7], cmul(s.w4, s.w3));
    }
    if constexpr (R >= 16) {
        v[8] = mul(v[8], s.w8);
        v[9] = mul(v[9], cmul(s.w8, s.w1));
        v[10] = mul(v[10], cmul(s.w8, s.w2));
        v[11] = mul(v[11], cmul(s.w8, s.w3));
        v[12] = mul(v[12], s.w12);
        v[13] = mul(v[13], cmul(s.w12, s.w1));
        v[14] = mul(v[14], cmul(s.w12, s.w2));
        v[15] = mul(v[15], cmul(s.w12, s.w3));
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
template <int L>
struct Lines {
    float2 *base;
    int lstride;
    __device__ __forceinline__ float2 ld(int l, int p) const { return base[l * lstride + padpos(p)]; }
    __device__ __forceinline__ void st(int l, int p, float2 v) const { base[l * lstride + padpos(p)] = v; }
};

// All twiddles a thread t needs for one transform of length M: one set per
// stage S > 0 and per butterfly q.  They depend on t only, so a thread can
// load them once and reuse them for every line, for both directions and for
// every tile it processes.
template <int M, int E>
struct ThreadTwiddles {
    using P = RadixPlan<M>;
    static constexpr int B1 = P::NS > 1 ? E / P::radix(P::NS > 1 ? 1 : 0) : 1;
    static constexpr int B2 = P::NS > 2 ? E / P::radix(P::NS > 2 ? 2 : 0) : 1;
    TwSet<P::radix(P::NS > 1 ? 1 : 0)> s1[B1];
    TwSet<P::radix(P::NS > 2 ? 2 : 0)> s2[B2];

    __device__ __forceinline__ void load(const float2 *__restrict__ tw, int t) {
        constexpr int T = M / E;
        if constexpr (P::NS > 1) {
            constexpr int R = P::radix(1), Ns = P::span(1);
#pragma unroll
            for (int q = 0; q < B1; q++) s1[q] = load_twiddles<R>(tw, ((t + q * T) & (Ns - 1)) * (M / (Ns * R)));
        }
        if constexpr (P::NS > 2) {
            constexpr int R = P::radix(2), Ns = P::span(2);
#pragma unroll
            for (int q = 0; q < B2; q++) s2[q] = load_twiddles<R>(tw, ((t + q * T) & (Ns - 1)) * (M / (Ns * R)));
        }
    }
    template <int S, int Q>
    __device__ __forceinline__ const auto &get() const {
        if constexpr (S == 1) return s1[Q];
        else return s2[Q];
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
template <int M, int E, int DIR, int S, int L, class TWS, class SYNC = BlockSync, bool WAR = true>
__device__ __forceinline__ void fft_stage(float2 (&a)[L][E], const Lines<L> &sm, int t,
                                          const float2 *__restrict__ tw, const TWS *twr,
                                          const SYNC &sync = SYNC()) {
    using P = RadixPlan<M>;
    constexpr int R = P::radix(S);
    constexpr int Ns = P::span(S);
    constexpr int B = E / R;
    constexpr int T = M / E;
    constexpr bool LAST = (S == P::NS - 1);
    static_assert(E % R == 0, "radix must divide E");
    if constexpr (S > 0) {
        sync();  // previous stage's outputs are in shared memory
#pragma unroll
        for (int l = 0; l < L; l++)
#pragma unroll
            for (int q = 0; q < B; q++)
#pragma unroll
                for (int r = 0; r < R; r++) a[l][q + r * B] = sm.ld(l, t + T * (q + r * B));
    }
    if constexpr (!LAST && WAR) sync();  // every read of this buffer is done
    static_for<B>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const int j = t + q * T;
        TwSet<R> ts;
        if constexpr (S > 0) {
            if constexpr (std::is_same<TWS, void>::value) ts = load_twiddles<R>(tw, (j & (Ns - 1)) * (M / (Ns * R)));
            else ts = twr->template get<S, q>();
        }
        const int base = (j / Ns) * Ns * R + (j & (Ns - 1));
#pragma unroll
        for (int l = 0; l < L; l++) {
            float2 v[R];
#pragma unroll
            for (int r = 0; r < R; r++) v[r] = a[l][q + r * B];
            if constexpr (S > 0) apply_twiddles<R, DIR>(v, ts);
            dft<R, DIR>(v);
            if constexpr (LAST) {
#pragma unroll
                for (int r = 0; r < R; r++) a[l][q + r * B] = v[r];
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
template <int M, int E, int DIR, int L, class TWS = void, class SYNC = BlockSync, bool FRESH = false>
__device__ __forceinline__ void fft_lines(float2 (&a)[L][E], const Lines<L> &sm, int t,
                                          const float2 *__restrict__ tw, const TWS *twr = nullptr,
                                          const SYNC &sync = SYNC()) {
    using P = RadixPlan<M>;
    static_assert(P::NS <= 3, "M up to 4096");
    fft_stage<M, E, DIR, 0, L, TWS, SYNC, !FRESH>(a, sm, t, tw, twr, sync);
    if constexpr (P::NS > 1) fft_stage<M, E, DIR, (P::NS > 1 ? 1 : 0), L, TWS, SYNC>(a, sm, t, tw, twr, sync);
    if constexpr (P::NS > 2) fft_stage<M, E, DIR, (P::NS > 2 ? 2 : 0), L, TWS, SYNC>(a, sm, t, tw, twr, sync);
}

}  // namespace tbs
