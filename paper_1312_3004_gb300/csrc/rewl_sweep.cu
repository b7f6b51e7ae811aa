// rewl_sweep.cu -- the fast WL sweep (Sec. 2 of arXiv:1312.3004) for sm_103a.
//
// Same arithmetic as the binary64 reference sweep in rewl_kernels.cu, bit for
// bit, organised for a GPU whose FP64 pipe is narrow and slow (GB300: one DADD
// has ~64 cycles of latency and ~2 per clock per SM of throughput):
//
//  * A group of S lanes (S = 1 .. 32, a power of two) owns one walker.  Each
//    lane prepares one of the next S proposals in parallel: Philox block,
//    site, new value, energy change against the lattice at the start of the
//    batch, and two integer acceptance thresholds.  The group then resolves the
//    S proposals in order; a proposal whose neighbourhood an earlier accepted
//    flip of the same batch touched is recomputed from the current lattice.
//  * ln g values are non-negative binary64 numbers, so their bit patterns
//    compare like the values.  D = bits(ln g(E')) - bits(ln g(E)) is the exact
//    difference in units of the last place when both lie in the same binade,
//    and "u < exp(ln g(E) - ln g(E'))" becomes D < T with T = -ln(u) / ulp.  T is
//    bracketed by [t_lo, t_hi) from a float estimate of -ln u with a proven
//    error margin; D < t_lo accepts and D >= t_hi rejects with certainty.  Only a
//    D inside the bracket (or operands in different binades) takes the
//    binary64 path exp(a - b) -- the same operation the reference performs.
//  * ln g(E) += ln f is an integer add of ln f / ulp to the bit pattern while
//    the sum stays in the binade (ln f = 2^-k is an exact multiple of the ulp);
//    otherwise a binary64 add.
//  * The current bin's ln g and visit count live in registers and are written
//    to shared memory when the walker leaves the bin.
#include <cstdint>

#include "rewl_internal.cuh"

namespace rewl {
namespace fast {

__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                        uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a0 = c0, a2 = c2;
        c0 = __umulhi(0xCD9E8D57u, a2) ^ c1 ^ k0;
        c2 = __umulhi(0xD2511F53u, a0) ^ c3 ^ k1;
        c1 = 0xCD9E8D57u * a2;
        c3 = 0xD2511F53u * a0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

template <int BITS>
__device__ __forceinline__ int spin_get(const uint32_t *w, int s) {
    if (BITS == 8) return reinterpret_cast<const uint8_t *>(w)[s];
    return (int)((w[s >> 3] >> ((s & 7) << 2)) & 15u);
}
template <int BITS>
__device__ __forceinline__ void spin_set(uint32_t *w, int s, int v) {
    if (BITS == 8) {
        reinterpret_cast<uint8_t *>(w)[s] = (uint8_t)v;
    } else {
        const uint32_t sh = (uint32_t)(s & 7) << 2;
        w[s >> 3] = (w[s >> 3] & ~(15u << sh)) | ((uint32_t)v << sh);
    }
}

struct Site4 { int r, l, d, u; };
__device__ __forceinline__ Site4 nbrs(int s, int L, int N, uint32_t divL) {
    const int y = (int)__umulhi((uint32_t)s, divL);
    const int x = s - y * L;
    Site4 n;
    n.r = (x == L - 1) ? s - (L - 1) : s + 1;
    n.l = (x == 0) ? s + (L - 1) : s - 1;
    n.d = (y == L - 1) ? s - (N - L) : s + L;
    n.u = (y == 0) ? s + (N - L) : s - L;
    return n;
}

template <int BITS>
__device__ __forceinline__ int energy_change(const uint32_t *lat, const Site4 &n, int cur, int nw) {
    const int a = spin_get<BITS>(lat, n.r), b = spin_get<BITS>(lat, n.l);
    const int c = spin_get<BITS>(lat, n.d), d = spin_get<BITS>(lat, n.u);
    return (int)(a == cur) + (int)(b == cur) + (int)(c == cur) + (int)(d == cur) - (int)(a == nw) -
           (int)(b == nw) - (int)(c == nw) - (int)(d == nw);
}

// 53-bit integer of the uniform u = U * 2^-53 (27 bits of hi, 26 of lo).
__device__ __forceinline__ unsigned long long u53(uint32_t hi, uint32_t lo) {
    return ((unsigned long long)(hi >> 5) << 26) | (lo >> 6);
}

constexpr long long kNoReject = 0x7fffffffffffffffLL;

// floor / ceil of x * 2^k as a 64-bit integer, saturating at 2^62 (x >= 0).
__device__ __forceinline__ long long scaled_floor(float x, int k) {
    if (x <= 0.0f) return 0;
    if (k > 120) return 1LL << 62;
    const float y = x * __int_as_float((k + 127) << 23);
    return y >= 0x1p62f ? (1LL << 62) : __float2ll_rd(y);
}
__device__ __forceinline__ long long scaled_ceil(float x, int k) {
    if (x <= 0.0f) return 0;
    if (k > 120) return 1LL << 62;
    const float y = x * __int_as_float((k + 127) << 23);
    return y >= 0x1p62f ? (1LL << 62) : __float2ll_ru(y);
}

// Bracket of T = -ln(u) / ulp(binade e0): accept-certain if D < t_lo,
// reject-certain if D >= t_hi.  uf = u with relative error <= 2^-23 (24 + 24
// bits, one rounding; top >= 1 makes the 5 dropped bits <= 2^-24 relative);
// logf is within 1 ulp; so |Lf - (-ln u)| <= (Lf + 1) 2^-22.9 and the margin
// (Lf + 1) 2^-18 leaves a factor > 8.  exp's own error (1 ulp of binary64)
// and the rounding of Lf -/+ margin are far inside that slack.
__device__ __forceinline__ void accept_bracket(unsigned long long U, int e0, long long &t_lo, long long &t_hi) {
    const uint32_t top = (uint32_t)(U >> 29);
    if (top == 0u || e0 == 0) {  // u < 2^-24, or no binade yet: decide exactly
        t_lo = 0;
        t_hi = kNoReject;
        return;
    }
    const float uf = fmaf((float)top, 0x1p-24f, (float)((uint32_t)(U >> 5) & 0xffffffu) * 0x1p-48f);
    const float Lf = -logf(uf);
    const float margin = (Lf + 1.0f) * 0x1p-18f;
    const int k = 1075 - e0;  // ulp = 2^(e0 - 1075)
    t_lo = scaled_floor(Lf - margin, k);
    t_hi = scaled_ceil(Lf + margin, k) + 1;
}

// Binade of a, and the integer step ln f / ulp(a) if it is exact.
struct Binade {
    long long lo, hi;  // [lo, hi) bit patterns with exponent e0
    long long inc;     // ln f in units of ulp(binade)
    int e0;
    bool add_ok;
};
__device__ __forceinline__ Binade binade_of(long long A, long long LNF) {
    Binade b;
    b.e0 = (int)(A >> 52);
    b.lo = (long long)b.e0 << 52;
    b.hi = (long long)(b.e0 + 1) << 52;
    b.inc = 0;
    b.add_ok = false;
    if (LNF == 0) {
        b.add_ok = true;
    } else if (b.e0 > 0 && (LNF >> 52) > 0) {
        const int el = (int)(LNF >> 52);
        const long long ml = (LNF & ((1LL << 52) - 1)) | (1LL << 52);
        const int sh = el - b.e0;
        if (sh >= 0) {
            if (sh <= 9) {
                b.inc = ml << sh;
                b.add_ok = b.inc < (1LL << 52);
            }
        } else if (sh > -53 && (ml & ((1LL << -sh) - 1)) == 0) {
            b.inc = ml >> -sh;
            b.add_ok = true;
        }
    }
    return b;
}

// The reference decision in binary64: accept iff D >= 0 or u < exp(D),
// D = a - b.
__device__ __noinline__ bool exact_accept(long long A, long long B, unsigned long long U, unsigned long long *ties) {
    const double d = __dsub_rn(__longlong_as_double(A), __longlong_as_double(B));
    if (d >= 0.0) return true;
    const double u = __ull2double_rn(U) * 0x1p-53;
    const double e = exp(d);
    if (fabs(u - e) < 1e-14) *ties += 1ull;
    return u < e;
}

__device__ __noinline__ long long exact_add(long long A, double lnf) {
    return __double_as_longlong(__dadd_rn(__longlong_as_double(A), lnf));
}

template <int S>
__device__ __forceinline__ unsigned group_mask() {
    if (S >= 32) return 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    return ((1u << (S & 31)) - 1u) << (lane & ~(unsigned)(S - 1));
}

// Per-walker scratch of the lane group in shared memory (S > 1 only).
struct Stage {
    unsigned long long *pk;  // [S] packed proposal
    long long *th;           // [2S] thresholds
    unsigned long long *uu;  // [S] 53-bit uniforms
    uint32_t *bm;            // [ceil(N/32)] sites touched by this batch
};

// packed proposal: site (20 bits) | v (8) << 20 | cur (8) << 28 | new (8) << 36 |
// (dE + 4) (4) << 44 | maybe-dirty (1) << 48
__device__ __forceinline__ unsigned long long pack(int site, int v, int cur, int nw, int dE, bool maybe) {
    return (unsigned long long)site | ((unsigned long long)v << 20) | ((unsigned long long)cur << 28) |
           ((unsigned long long)nw << 36) | ((unsigned long long)(dE + 4) << 44) |
           ((unsigned long long)(maybe ? 1 : 0) << 48);
}

struct Tally {
    unsigned long long acc, ties, slow;
};

template <int BITS, int S>
__device__ void walker_sweep(const Model &M, uint32_t *lat, double *lg, uint32_t *hg, const Stage &st, int g, int lo,
                             double lnf, int &E_io, unsigned long long &t_io, Tally &tally) {
    const int j = (int)(threadIdx.x & (unsigned)(S - 1));
    const unsigned gm = group_mask<S>();
    const int W = M.W, N = M.N, L = M.L;
    const uint32_t qm1 = (uint32_t)(M.q - 1);
    const long long LNF = __double_as_longlong(lnf);
    int E = E_io;
    unsigned long long t = t_io;
    long long A = __double_as_longlong(lg[E - lo]);
    uint32_t visits = 0;
    Binade bn = binade_of(A, LNF);

    for (long long base = 0; base < M.K; base += S) {
        const int n = (int)((M.K - base) < S ? (M.K - base) : S);
        // ---- parallel phase: lane j prepares proposal t + j ------------------
        int site = N + j, v = 0, cur = 0, nw = 0, dE = 0;
        Site4 nb{0, 0, 0, 0};
        long long tlo = 0, thi = kNoReject;
        unsigned long long U = 0;
        if (j < n) {
            const unsigned long long tj = t + (unsigned long long)j;
            const uint4 r = philox((uint32_t)tj, (uint32_t)(tj >> 32), (uint32_t)g, DOM_WL, M.key0, M.key1);
            site = (int)__umulhi(r.x, (uint32_t)N);
            v = (int)__umulhi(r.y, qm1);
            cur = spin_get<BITS>(lat, site);
            nw = v + (v >= cur);
            nb = nbrs(site, L, N, M.divL);
            dE = energy_change<BITS>(lat, nb, cur, nw);
            U = u53(r.z, r.w);
            accept_bracket(U, bn.e0, tlo, thi);
        }
        if (S == 1) {
            // ---- single lane: resolve directly --------------------------------
            if (j < n) {
                const int En = E + dE;
                bool acc = false;
                long long B = A;
                if ((unsigned)(En - lo) <= (unsigned)W) {
                    if (En == E) {
                        acc = true;
                    } else {
                        B = __double_as_longlong(lg[En - lo]);
                        if (B <= A) {
                            acc = true;
                        } else {
                            const long long D = B - A;
                            const bool fast = A >= bn.lo && B < bn.hi;
                            if (fast && D < tlo) acc = true;
                            else if (fast && D >= thi) acc = false;
                            else {
                                tally.slow += 1;
                                acc = exact_accept(A, B, U, &tally.ties);
                            }
                        }
                    }
                }
                if (acc) {
                    spin_set<BITS>(lat, site, nw);
                    tally.acc += 1;
                    if (En != E) {
                        lg[E - lo] = __longlong_as_double(A);
                        hg[E - lo] += visits;
                        E = En;
                        A = B;
                        visits = 0;
                    }
                }
                const long long A2 = A + bn.inc;
                if (bn.add_ok && A >= bn.lo && A2 < bn.hi) A = A2;
                else A = exact_add(A, lnf);
                visits += 1;
            }
        } else {
            // ---- conflict marks: sites proposed in this batch -----------------
            if (j < n) atomicOr(&st.bm[site >> 5], 1u << (site & 31));
            __syncwarp(gm);
            const unsigned peers = __match_any_sync(gm, site);
            const unsigned lane = threadIdx.x & 31u;
            bool maybe = (peers & ((1u << lane) - 1u) & gm) != 0u;
            if (j < n) {
                maybe |= ((st.bm[nb.r >> 5] >> (nb.r & 31)) | (st.bm[nb.l >> 5] >> (nb.l & 31)) |
                          (st.bm[nb.d >> 5] >> (nb.d & 31)) | (st.bm[nb.u >> 5] >> (nb.u & 31))) & 1u;
                st.pk[j] = pack(site, v, cur, nw, dE, maybe);
                st.th[2 * j] = tlo;
                st.th[2 * j + 1] = thi;
                st.uu[j] = U;
            }
            __syncwarp(gm);
            if (j < n) st.bm[site >> 5] = 0u;  // every marked word belongs to some lane's site
            // ---- serial phase: the group resolves the proposals in order -------
            bool any_acc = false;
            for (int k = 0; k < n; ++k) {
                const unsigned long long pk = st.pk[k];
                int ks = (int)(pk & 0xfffffu);
                int knw = (int)((pk >> 36) & 0xffu);
                int kdE = (int)((pk >> 44) & 0xfu) - 4;
                if (((pk >> 48) & 1ull) && any_acc) {  // neighbourhood changed in this batch
                    const int kv = (int)((pk >> 20) & 0xffu);
                    const int kc = spin_get<BITS>(lat, ks);
                    knw = kv + (kv >= kc);
                    kdE = energy_change<BITS>(lat, nbrs(ks, L, N, M.divL), kc, knw);
                }
                const int En = E + kdE;
                bool acc = false;
                long long B = A;
                if ((unsigned)(En - lo) <= (unsigned)W) {
                    if (En == E) {
                        acc = true;
                    } else {
                        B = __double_as_longlong(lg[En - lo]);
                        if (B <= A) {
                            acc = true;
                        } else {
                            const long long D = B - A;
                            const bool fast = A >= bn.lo && B < bn.hi;
                            const long long klo = st.th[2 * k], khi = st.th[2 * k + 1];
                            if (fast && D < klo) acc = true;
                            else if (fast && D >= khi) acc = false;
                            else {
                                tally.slow += 1;
                                acc = exact_accept(A, B, st.uu[k], &tally.ties);
                            }
                        }
                    }
                }
                if (acc) {
                    spin_set<BITS>(lat, ks, knw);
                    any_acc = true;
                    tally.acc += 1;
                    if (En != E) {
                        lg[E - lo] = __longlong_as_double(A);
                        if (j == 0) hg[E - lo] += visits;
                        E = En;
                        A = B;
                        visits = 0;
                    }
                }
                const long long A2 = A + bn.inc;
                if (bn.add_ok && A >= bn.lo && A2 < bn.hi) A = A2;
                else A = exact_add(A, lnf);
                visits += 1;
            }
            __syncwarp(gm);
        }
        t += (unsigned long long)n;
        if ((A >> 52) != bn.e0) bn = binade_of(A, LNF);
    }
    lg[E - lo] = __longlong_as_double(A);
    if (j == 0) hg[E - lo] += visits;
    E_io = E;
    t_io = t;
}

// Shared-memory layout of one walker.
struct Layout {
    int stride;           // bytes per walker (multiple of 16)
    int off_H, off_lat;   // byte offsets (ln g at 0)
    int off_pk, off_th, off_uu, off_bm;
};

template <int BITS, int S>
__global__ void __launch_bounds__(256) sweep_fast_kernel(Model M, State Sg, int P, Layout lay) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (*(volatile unsigned int *)&Sg.ctl->all_done) return;
    const int g0 = blockIdx.x * P;
    for (int p = 0; p < P; ++p) {
        const int g = g0 + p;
        if (g >= M.G || Sg.done[g / M.m]) continue;
        unsigned char *base = smem + (size_t)p * lay.stride;
        double *lg = reinterpret_cast<double *>(base);
        uint32_t *hg = reinterpret_cast<uint32_t *>(base + lay.off_H);
        uint32_t *lat = reinterpret_cast<uint32_t *>(base + lay.off_lat);
        const double *src_lg = Sg.lng + (size_t)g * M.B;
        const uint32_t *src_H = Sg.H + (size_t)g * M.B;
        const uint32_t *src_lat = Sg.spins + (size_t)Sg.slot_cfg[g] * M.wpc;
        for (int i = threadIdx.x; i < M.B; i += blockDim.x) {
            lg[i] = src_lg[i];
            hg[i] = src_H[i];
        }
        for (int i = threadIdx.x; i < M.wpc; i += blockDim.x) lat[i] = src_lat[i];
        if (S > 1) {
            uint32_t *bm = reinterpret_cast<uint32_t *>(base + lay.off_bm);
            for (int i = threadIdx.x; i < (M.N + 31) / 32; i += blockDim.x) bm[i] = 0u;
        }
    }
    __syncthreads();

    const int grp = threadIdx.x / S, g = g0 + grp;
    Tally tally{0ull, 0ull, 0ull};
    if (grp < P && g < M.G && !Sg.done[g / M.m]) {
        unsigned char *base = smem + (size_t)grp * lay.stride;
        Stage st;
        st.pk = reinterpret_cast<unsigned long long *>(base + lay.off_pk);
        st.th = reinterpret_cast<long long *>(base + lay.off_th);
        st.uu = reinterpret_cast<unsigned long long *>(base + lay.off_uu);
        st.bm = reinterpret_cast<uint32_t *>(base + lay.off_bm);
        const int w = g / M.m;
        const uint32_t c = Sg.slot_cfg[g];
        int E = Sg.cfg_E[c];
        unsigned long long t = Sg.t[g];
        walker_sweep<BITS, S>(M, reinterpret_cast<uint32_t *>(base + lay.off_lat), reinterpret_cast<double *>(base),
                              reinterpret_cast<uint32_t *>(base + lay.off_H), st, g, Sg.e_lo[w], Sg.lnf[w], E, t,
                              tally);
        if ((threadIdx.x & (S - 1)) == 0) {
            Sg.cfg_E[c] = E;
            Sg.t[g] = t;
            atomicAdd(&Sg.ctl->flips, (unsigned long long)M.K);
            atomicAdd(&Sg.ctl->accepted, tally.acc);
            if (tally.slow) atomicAdd(&Sg.ctl->slow, tally.slow);
            if (tally.ties) atomicAdd(&Sg.ctl->ties, tally.ties);
        }
    }
    __syncthreads();

    for (int p = 0; p < P; ++p) {
        const int gg = g0 + p;
        if (gg >= M.G || Sg.done[gg / M.m]) continue;
        const unsigned char *base = smem + (size_t)p * lay.stride;
        const double *lg = reinterpret_cast<const double *>(base);
        const uint32_t *hg = reinterpret_cast<const uint32_t *>(base + lay.off_H);
        const uint32_t *lat = reinterpret_cast<const uint32_t *>(base + lay.off_lat);
        double *dst_lg = Sg.lng + (size_t)gg * M.B;
        uint32_t *dst_H = Sg.H + (size_t)gg * M.B;
        uint32_t *dst_lat = Sg.spins + (size_t)Sg.slot_cfg[gg] * M.wpc;
        for (int i = threadIdx.x; i < M.B; i += blockDim.x) {
            dst_lg[i] = lg[i];
            dst_H[i] = hg[i];
        }
        for (int i = threadIdx.x; i < M.wpc; i += blockDim.x) dst_lat[i] = lat[i];
    }
}

Layout make_layout(const Model &M, int S) {
    auto al = [](int x) { return (x + 15) & ~15; };
    Layout l{};
    int off = al(M.B * 8);
    l.off_H = off;
    off += al(M.B * 4);
    l.off_lat = off;
    off += al(M.wpc * 4);
    if (S > 1) {
        l.off_pk = off;
        off += al(S * 8);
        l.off_th = off;
        off += al(S * 16);
        l.off_uu = off;
        off += al(S * 8);
        l.off_bm = off;
        off += al(((M.N + 31) / 32) * 4);
    }
    l.stride = al(off);
    return l;
}

template <int BITS, int S>
cudaError_t launch_t(const Model &M, const State &St, const SweepPlan &p, cudaStream_t s, bool prepare) {
    const Layout lay = make_layout(M, S);
    if (prepare)
        return cudaFuncSetAttribute(sweep_fast_kernel<BITS, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)p.smem);
    sweep_fast_kernel<BITS, S><<<p.grid, p.threads, p.smem, s>>>(M, St, p.P, lay);
    return cudaGetLastError();
}

template <int BITS>
cudaError_t dispatch_s(const Model &M, const State &St, const SweepPlan &p, cudaStream_t s, bool prepare) {
    switch (p.lanes) {
    case 1: return launch_t<BITS, 1>(M, St, p, s, prepare);
    case 2: return launch_t<BITS, 2>(M, St, p, s, prepare);
    case 4: return launch_t<BITS, 4>(M, St, p, s, prepare);
    case 8: return launch_t<BITS, 8>(M, St, p, s, prepare);
    case 16: return launch_t<BITS, 16>(M, St, p, s, prepare);
    default: return launch_t<BITS, 32>(M, St, p, s, prepare);
    }
}

}  // namespace fast

size_t fast_smem_per_walker(const Model &M, int lanes) { return (size_t)fast::make_layout(M, lanes).stride; }

cudaError_t launch_sweep_fast(const Model &M, const State &S, const SweepPlan &p, cudaStream_t s, bool prepare) {
    return M.bits == 8 ? fast::dispatch_s<8>(M, S, p, s, prepare) : fast::dispatch_s<4>(M, S, p, s, prepare);
}

}  // namespace rewl
