// rewl_sweep.cu -- the fast WL sweep (Sec. 2 of arXiv:1312.3004) for sm_103a.
//
// Same states as the binary64 reference sweep in rewl_kernels.cu, bit for
// bit, organised for a GPU whose FP64 pipe is narrow and slow (GB300: one DADD
// has ~64 cycles of latency and ~2 per clock per SM of throughput):
//
//  * A group of S lanes (S = 1 .. 32, a power of two) owns one walker.  Each
//    lane prepares one of the next S proposals in parallel: Philox block,
//    site, new value, energy change against the lattice at the start of the
//    batch, and an integer acceptance bracket.  Proposals whose neighbourhood
//    another proposal of the batch touches are flagged.
//  * Tagged fixed-point shadow of ln g: for the launch, every ln g value v of
//    the walker is also held as F(v) = 2 floor(v / u) + (1 if the floor
//    dropped bits), u = 2^(e_w - 1075), e_w seven binades below the largest
//    value the launch can reach.  D = F(ln g(E')) - F(ln g(E)) is within three
//    half-units of the true difference, and the reference test
//    "u_rnd < exp(ln g(E) - ln g(E'))" is decided by D < T_lo (accept) or
//    D >= T_hi (reject), with [T_lo, T_hi) bracketing -ln(u_rnd) with a proven
//    margin.  Only D inside the bracket (about 1e-6 of the decisions) takes
//    the binary64 path exp(a - b) -- the operation the reference does.
//  * ln g(E) += ln f is an integer add on the shadow (ln f = 2^-k is a whole
//    number of half-units), rounded to 53 bits in integers when it enters the
//    next binade; values whose shadow dropped bits take binary64 steps.
//  * The group resolves the proposals of a batch by a tree of speculative
//    steps: lane j decides node j of the binary tree of the next log2(S)
//    steps from the state at the start of the window, and ballots follow the
//    true path.  Lattice writes and the visit histogram are applied in
//    parallel after the batch.
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

// Upper bracket end that never rejects inside a window (in-window |D| < 2^62).
constexpr long long kNoReject = 1LL << 62;
// Shadow value of the bins beyond each end of a window: every proposal there
// has D >= 2^62 >= t_hi and is rejected like an out-of-window move.  The
// padding also covers the loads of speculative paths (up to six moves of up
// to four bins each, see the step tree below).
constexpr long long kOutside = 0x7fffffffffffffffLL;
constexpr int kPad = kShadowPad;
constexpr long long kMant = (1LL << 52) - 1, kHidden = 1LL << 52;

// floor / ceil of x * 2^k as a 64-bit integer, saturating at 2^61 (x >= 0).
__device__ __forceinline__ long long scaled_floor(float x, int k) {
    if (x <= 0.0f) return 0;
    if (k > 120) return 1LL << 61;
    const float y = x * __int_as_float((k + 127) << 23);
    return y >= 0x1p61f ? (1LL << 61) : __float2ll_rd(y);
}
__device__ __forceinline__ long long scaled_ceil(float x, int k) {
    if (x <= 0.0f) return 0;
    if (k > 120) return 1LL << 61;
    const float y = x * __int_as_float((k + 127) << 23);
    return y >= 0x1p61f ? (1LL << 61) : __float2ll_ru(y);
}

// Bracket of T = -ln(u) / unit, unit = 2^-k: accept for sure if D < t_lo,
// reject for sure if D >= t_hi, where D is within three units of the true
// difference (the shadow's floors and inexact tags, see shadow_of).  uf = u with relative error <= 2^-23 (24 + 24 bits, one
// rounding; top >= 1 makes the 5 dropped bits <= 2^-24 relative); logf is
// within 1 ulp; so |Lf - (-ln u)| <= (Lf + 1) 2^-22.9, and the margin
// (Lf + 1) 2^-18 leaves a factor > 8 for that, for exp's own error (1 ulp of
// binary64) and for the rounding of Lf -/+ margin.
__device__ __forceinline__ void accept_bracket(unsigned long long U, int k, long long &t_lo, long long &t_hi) {
    const uint32_t top = (uint32_t)(U >> 29);
    if (top == 0u) {  // u < 2^-24: only D < 0 is decided here
        t_lo = 0;
        t_hi = kNoReject;
        return;
    }
    const float uf = fmaf((float)top, 0x1p-24f, (float)((uint32_t)(U >> 5) & 0xffffffu) * 0x1p-48f);
    const float Lf = -logf(uf);
    const float margin = (Lf + 1.0f) * 0x1p-18f;
    const long long lo = scaled_floor(Lf - margin, k) - 3;
    t_lo = lo > 0 ? lo : 0;
    t_hi = scaled_ceil(Lf + margin, k) + 4;
}

// Shadow of a non-negative binary64 bit pattern v in half-units of
// u = 2^(ew - 1075): 2 floor(v / u) + (1 if the floor dropped bits).  A value
// whose tag bit is 0 is exactly (shadow / 2) u.  The exponent of v is at most
// ew + 8, so the shadow stays below 2^62.
__device__ __forceinline__ long long shadow_of(long long v, int ew) {
    if (v == 0) return 0;
    const int s = (int)(v >> 52) - ew;
    const long long mf = (v & kMant) | kHidden;
    if (s >= 0) return (mf << s) << 1;
    if (s <= -53) return 1;
    return ((mf >> -s) << 1) | (long long)((mf & ((1LL << -s) - 1)) != 0);
}

// v / 2^(e - 1075) for the binary64 value v = ln f if that is an integer below
// 2^52 (ln f is an exact multiple of the unit and one step cannot span a
// binade); ok = false otherwise.
__device__ __forceinline__ long long exact_units(long long v, int e, bool &ok) {
    ok = true;
    if (v == 0) return 0;
    const int el = (int)(v >> 52);
    if (el == 0 || e <= 0) {
        ok = false;
        return 0;
    }
    const long long mf = (v & kMant) | kHidden;
    const int s = el - e;
    if (s >= 0) {
        if (s > 9) {
            ok = false;
            return 0;
        }
        const long long r = mf << s;
        ok = r < (1LL << 52);
        return r;
    }
    if (s <= -53 || (mf & ((1LL << -s) - 1)) != 0) {
        ok = false;
        return 0;
    }
    return mf >> -s;
}

// The reference decision in binary64: accept iff d >= 0 or u < exp(d), d = a - b.
// A draw with |u - exp(d)| < 1e-14 is a near tie: counted, and its step index
// kept (the first two of the walker's launch) for the tie log.
struct TieRec {
    unsigned long long n, t[2];
};
__device__ __noinline__ bool exact_accept(long long A, long long B, unsigned long long U, TieRec *tie,
                                          unsigned long long step) {
    const double d = __dsub_rn(__longlong_as_double(A), __longlong_as_double(B));
    if (d >= 0.0) return true;
    const double u = __ull2double_rn(U) * 0x1p-53;
    const double e = exp(d);
    if (fabs(u - e) < 1e-14) {
        if (tie->n < 2ull) tie->t[tie->n] = step;
        tie->n += 1ull;
    }
    return u < e;
}

// The walker's near ties of this launch into the control block and the log.
__device__ __forceinline__ void flush_ties(const State &S, int g, const TieRec &tie) {
    if (!tie.n) return;
    for (unsigned long long i = 0; i < tie.n && i < 2ull; ++i) record_tie(S.ctl, S.tlog, TIE_WL, (unsigned int)g, tie.t[i]);
    if (tie.n > 2ull) atomicAdd(&S.ctl->ties, tie.n - 2ull);
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
    longlong2 *q;  // [S + kStagePad] bracket of proposal k as the serial loop reads it: (t_lo, t_hi - t_lo)
    int *e;        // [S + kStagePad] energy change of proposal k as a byte step over the ln g shadow (8 dE)
    uint32_t *bm;    // [2 nbw] marks of the sites proposed in this batch; then of those proposed twice
    int nbw;         // ceil(min(N, kMarkBits) / 32)
    uint32_t mmask;  // site -> mark: all bits when N <= kMarkBits, else kMarkBits - 1 (shared marks
                     // only ever flag more proposals, never fewer)
};
constexpr int kStagePad = 8;
constexpr int kMarkBits = 8192;

// A bracket no difference passes: the serial loop hands the proposal to the
// exact step (t_lo below every in-window D, width covering every D).
constexpr long long kForceLo = -(1LL << 62);

struct Tally {
    TieRec tie;
    unsigned long long slow;
    unsigned int acc, seq;
#ifdef REWL_DEBUG_CHECKS
    unsigned int bad = 0;  // failed bounds checks
#endif
};

// Binary64 bits of F * 2^(ew - 1075) for an integer F >= 0 that has at most
// 53 significant bits (a value the shadow holds exactly).
__device__ __forceinline__ long long from_units(long long F, int ew) {
    if (F == 0) return 0;
    const int sh = 11 - __clzll(F);  // top bit position - 52
    const long long m = sh >= 0 ? (F >> sh) : (F << -sh);
    return ((long long)(ew + sh) << 52) | (m & kMant);
}

// Round an exact shadow (tag 0) to 53 significant bits, ties to even: the
// binary64 rounding of a ln f step that entered the next binade.
__device__ __forceinline__ long long round_shadow(long long F2) {
    long long F = F2 >> 1;
    const int sh = 11 - __clzll(F);
    if (sh <= 0) return F2;
    const long long ulp = 1LL << sh, r = F & (ulp - 1);
    if (r == 0) return F2;
    const long long half = ulp >> 1;
    F -= r;
    if (r > half || (r == half && ((F >> sh) & 1))) F += ulp;
    return F << 1;
}

// 64-bit access to the shadow array by 32-bit shared address.  Lanes of a
// group see each other's writes only across a __syncwarp.
__device__ __forceinline__ long long lds64(uint32_t a) {
    return *reinterpret_cast<const long long *>(__cvta_shared_to_generic(a));
}
__device__ __forceinline__ void sts64(uint32_t a, long long v) {
    *reinterpret_cast<long long *>(__cvta_shared_to_generic(a)) = v;
}

template <int S, typename T>
__device__ __forceinline__ T from_lane(unsigned gm, T x, int k) {
    if (S == 1) return x;
    return __shfl_sync(gm, x, k, S);
}

// One lane per walker: the steps one after another, each proposal drawn (and
// its spins read) while the previous step waits for its ln g shadow; a
// proposal whose site or neighbours the previous step flipped is re-read.
// The frame, the shadow, the bracket and the exact fallbacks are those of
// walker_sweep below.
template <int BITS>
__device__ void walker_sweep_1(const Model &M, uint32_t *__restrict__ lat, long long *__restrict__ lgb, long long *lgf,
                               uint32_t *__restrict__ hg, int g, int lo, double lnf, int &E_io,
                               unsigned long long &t_io, Tally &tally) {
    const int N = M.N, L = M.L;
    constexpr int per = 32 / BITS;
    const uint32_t qm1 = (uint32_t)(M.q - 1);
    const long long LNF = __double_as_longlong(lnf);
    long long vmax = 0;
    for (int b = 0; b < M.B; ++b) vmax = max(vmax, lgb[b]);
    const double reach = __dadd_rn(__longlong_as_double(vmax), __dmul_rn((double)M.K, lnf));
    int ew = (int)(__double_as_longlong(reach) >> 52) - 7;
    if (ew < 1) ew = 1;
    const int k = 1076 - ew;
    for (int b = 0; b < M.B; ++b) lgf[b] = shadow_of(lgb[b], ew);
    for (int p = 0; p < kPad; ++p) {
        lgf[-1 - p] = kOutside;
        lgf[M.B + p] = kOutside;
    }
    bool addF;
    const long long incU = exact_units(LNF, ew, addF);
    const long long incF = incU << 1;
    const bool int_add = addF && (incU & 255) == 0;

    struct Prop {
        int site, v, cur, sr, sl, sd, su;
        Site4 nb;
        longlong2 th;
        unsigned long long U;
    };
    auto draw = [&](unsigned long long tt, Prop &p) {
        const uint4 r = philox((uint32_t)tt, (uint32_t)(tt >> 32), (uint32_t)g, DOM_WL, M.key0, M.key1);
        p.site = (int)__umulhi(r.x, (uint32_t)N);
        p.v = (int)__umulhi(r.y, qm1);
        p.nb = nbrs(p.site, L, N, M.divL);
        p.cur = spin_get<BITS>(lat, p.site);
        p.sr = spin_get<BITS>(lat, p.nb.r);
        p.sl = spin_get<BITS>(lat, p.nb.l);
        p.sd = spin_get<BITS>(lat, p.nb.d);
        p.su = spin_get<BITS>(lat, p.nb.u);
        p.U = u53(r.z, r.w);
        accept_bracket(p.U, k, p.th.x, p.th.y);
    };
    // The current bin's shadow AF and its visits since the walker came are kept
    // in registers, and written when the walker leaves the bin.
    int Eo = E_io - lo;
    long long AF = lgf[REWL_IDX(Eo, 0, M.B, tally.bad)];
    uint32_t visits = 0;
    unsigned int nacc = 0;
    int flipped = -1;  // site the previous step flipped
    Prop cp;
    draw(t_io, cp);
    for (long long i = 0; i < M.K; ++i) {
        if (flipped >= 0 && (flipped == cp.site || flipped == cp.nb.r || flipped == cp.nb.l || flipped == cp.nb.d ||
                             flipped == cp.nb.u)) {
            cp.cur = spin_get<BITS>(lat, cp.site);
            cp.sr = spin_get<BITS>(lat, cp.nb.r);
            cp.sl = spin_get<BITS>(lat, cp.nb.l);
            cp.sd = spin_get<BITS>(lat, cp.nb.d);
            cp.su = spin_get<BITS>(lat, cp.nb.u);
        }
        const int nw = cp.v + (cp.v >= cp.cur);
        const int dE = (int)(cp.sr == cp.cur) + (int)(cp.sl == cp.cur) + (int)(cp.sd == cp.cur) + (int)(cp.su == cp.cur) -
                       (int)(cp.sr == nw) - (int)(cp.sl == nw) - (int)(cp.sd == nw) - (int)(cp.su == nw);
        const int En = Eo + dE;
        const long long BF = dE == 0 ? AF : lgf[REWL_IDX(En, -kPad, M.B + kPad, tally.bad)];  // beyond: kOutside
        Prop np;
        if (i + 1 < M.K) draw(t_io + (unsigned long long)i + 1ull, np);
        const long long D = BF - AF;
        bool acc = D < cp.th.x;
        if (!acc && D < cp.th.y) {  // inside the bracket (never beyond the window)
            tally.slow += 1;
            const long long Ab = (AF & 1) ? lgb[REWL_IDX(Eo, 0, M.B, tally.bad)] : from_units(AF >> 1, ew);
            const long long Bb = (BF & 1) ? lgb[REWL_IDX(En, 0, M.B, tally.bad)] : from_units(BF >> 1, ew);
            acc = dE == 0 ? true : exact_accept(Ab, Bb, cp.U, &tally.tie, t_io + (unsigned long long)i);
        }
        const long long cur = acc ? BF : AF;  // with dE = 0 both are the current shadow
        const int Eb2 = acc ? En : Eo;
        long long AF2 = cur + incF;
        if (!int_add || (cur & 1)) {  // ln g(E) += ln f in binary64
            tally.seq += 1;
            const long long Ab = (cur & 1) ? lgb[REWL_IDX(Eb2, 0, M.B, tally.bad)] : from_units(cur >> 1, ew);
            const long long A2 = exact_add(Ab, lnf);
            lgb[REWL_IDX(Eb2, 0, M.B, tally.bad)] = A2;
            AF2 = shadow_of(A2, ew);
        } else {
            const uint32_t hc = (uint32_t)((unsigned long long)cur >> 32);
            const uint32_t h2 = (uint32_t)((unsigned long long)AF2 >> 32);
            if ((h2 ^ hc) > hc) AF2 = round_shadow(AF2);  // into the next binade
        }
        // (atomics whose result is not used: the walker does not wait for them)
        if (Eb2 != Eo) {  // leaving the bin: its value and visits go to memory
            lgf[REWL_IDX(Eo, 0, M.B, tally.bad)] = AF;
            atomicAdd(&hg[REWL_IDX(Eo, 0, M.B, tally.bad)], visits);
            visits = 0;
        }
        ++visits;
        Eo = Eb2;
        AF = AF2;
        if (acc) {
            atomicXor(&lat[cp.site / per], (uint32_t)(cp.cur ^ nw) << ((cp.site & (per - 1)) * BITS));
            ++nacc;
        }
        flipped = acc ? cp.site : -1;
        cp = np;
    }
    lgf[Eo] = AF;
    atomicAdd(&hg[Eo], visits);
    t_io += (unsigned long long)M.K;
    for (int b = 0; b < M.B; ++b) {
        const long long F = lgf[b];
        if (!(F & 1)) lgb[b] = from_units(F >> 1, ew);
    }
    tally.acc += nacc;
    E_io = Eo + lo;
}

template <int BITS, int S>
__device__ void walker_sweep(const Model &M, uint32_t *__restrict__ lat, long long *__restrict__ lgb,
                             long long *lgf, uint32_t *__restrict__ hg, const Stage &st, int g, int lo,
                             double lnf, int &E_io, unsigned long long &t_io, Tally &tally) {
    if constexpr (S == 1) {
        walker_sweep_1<BITS>(M, lat, lgb, lgf, hg, g, lo, lnf, E_io, t_io, tally);
        return;
    }
    const int j = (int)(threadIdx.x & (unsigned)(S - 1));
    const unsigned gm = group_mask<S>();
    const int N = M.N, L = M.L;
    constexpr int per = 32 / BITS;  // sites per lattice word
    const uint32_t qm1 = (uint32_t)(M.q - 1);
    const long long LNF = __double_as_longlong(lnf);

    // ---- fixed-point frame of this launch --------------------------------------
    long long vmax = 0;
    for (int b = j; b < M.B; b += S) vmax = max(vmax, lgb[b]);
#pragma unroll
    for (int o = 1; o < S; o <<= 1) vmax = max(vmax, __shfl_xor_sync(gm, vmax, o));
    const double reach = __dadd_rn(__longlong_as_double(vmax), __dmul_rn((double)M.K, lnf));
    // values stay below 2^(e_reach + 2 - 1023): below 2^61 units of
    // u = 2^(ew - 1075), shadows (half-units) below 2^62
    int ew = (int)(__double_as_longlong(reach) >> 52) - 7;
    if (ew < 1) ew = 1;
    const int k = 1076 - ew;  // half-unit = 2^-k
    for (int b = j; b < M.B; b += S) lgf[b] = shadow_of(lgb[b], ew);
    for (int p = j; p < kPad; p += S) {
        lgf[-1 - p] = kOutside;
        lgf[M.B + p] = kOutside;
    }
    bool addF;
    const long long incU = exact_units(LNF, ew, addF);
    const long long incF = incU << 1;  // ln f in half-units
    // every integer step inside a binade is exact when ln f is a multiple of the
    // largest last place (2^8 units for values below 2^61 units)
    const bool int_add = addF && (incU & 255) == 0;
    if (S > 1) __syncwarp(gm);

    // The current bin: Eo its index in the window, AF its shadow (always equal
    // to lgf[Eo]), pcur the shared address of lgf[Eo].  A shadow >= 2^52 is the
    // value exactly; below that the exact binary64 bits are kept in lgb.
    int Eo = E_io - lo;
    // (lane groups: the shadow is in shared memory; one lane: shared or global)
    const uint32_t pbase = S > 1 ? (uint32_t)__cvta_generic_to_shared(lgf) : 0u;
    long long AF = lgf[Eo];
    unsigned int nacc = 0;
    // node of this lane in the step tree (lane S - 1 has none)
    constexpr int DP = S >= 32 ? 5 : S >= 16 ? 4 : S >= 8 ? 3 : S >= 4 ? 2 : 1;
    const int lvl = 31 - __clz(j + 1), pre = j + 1 - (1 << lvl);
    const unsigned lane = threadIdx.x & 31u, gbase = lane & ~(unsigned)(S - 1);
    // its ancestors, (l, pre mod 2^l) at node index 2^l - 1 + (pre mod 2^l): which
    // they are, and the decision each must take for the path to lead here
    unsigned anc_mask = 0u, anc_bits = 0u;
    bool tl[DP > 1 ? DP - 1 : 1], tb[DP > 1 ? DP - 1 : 1];  // step l on the path; taken as a move
#pragma unroll
    for (int l = 0; l < DP - 1; ++l) {
        tl[l] = l < lvl;
        tb[l] = l < lvl && ((pre >> l) & 1);
        if (l < lvl) {
            const int a = (1 << l) - 1 + (pre & ((1 << l) - 1));
            anc_mask |= 1u << a;
            anc_bits |= (unsigned)((pre >> l) & 1) << a;
        }
    }

    for (long long base = 0; base < M.K; base += S) {
        const int n = (int)((M.K - base) < S ? (M.K - base) : S);
        // ---- parallel phase: lane j prepares proposal t + j --------------------
        int site = N + j, v = 0, dE = 0, word = 0;
        Site4 nb{0, 0, 0, 0};
        uint32_t xr = 0;  // the flip as an xor on its lattice word
        longlong2 th = make_longlong2(0, kNoReject);
        unsigned long long U = 0;
        if (j < n) {
            const unsigned long long tj = t_io + (unsigned long long)j;
            const uint4 r = philox((uint32_t)tj, (uint32_t)(tj >> 32), (uint32_t)g, DOM_WL, M.key0, M.key1);
            site = (int)__umulhi(r.x, (uint32_t)N);
            v = (int)__umulhi(r.y, qm1);
            const int cur = spin_get<BITS>(lat, site);
            const int nw = v + (v >= cur);
            nb = nbrs(site, L, N, M.divL);
            dE = energy_change<BITS>(lat, nb, cur, nw);
            word = site / per;
            xr = (uint32_t)(cur ^ nw) << ((site & (per - 1)) * BITS);
            U = u53(r.z, r.w);
            accept_bracket(U, k, th.x, th.y);
        }
        bool flag = false;  // an earlier proposal of the batch may change dE
        longlong2 q1 = make_longlong2(th.x, th.y - th.x);
        if (S > 1) {
            // ---- conflict marks: sites proposed in this batch -------------------
            // (a site proposed twice marks both proposals: the later one needs it)
            const uint32_t ms = (uint32_t)site & st.mmask;
            const int wsite = (int)(ms >> 5);
            const uint32_t bsite = 1u << (ms & 31);
            uint32_t *dup = st.bm + st.nbw;
            if (j < n && (atomicOr(&st.bm[wsite], bsite) & bsite)) atomicOr(&dup[wsite], bsite);
            __syncwarp(gm);
            if (j < n) {
                const uint32_t mr = (uint32_t)nb.r & st.mmask, ml = (uint32_t)nb.l & st.mmask;
                const uint32_t md = (uint32_t)nb.d & st.mmask, mu = (uint32_t)nb.u & st.mmask;
                flag = ((dup[wsite] >> (ms & 31)) | (st.bm[mr >> 5] >> (mr & 31)) | (st.bm[ml >> 5] >> (ml & 31)) |
                        (st.bm[md >> 5] >> (md & 31)) | (st.bm[mu >> 5] >> (mu & 31))) & 1u;
                st.q[j] = flag ? make_longlong2(kForceLo, -1LL) : q1;
                st.e[j] = dE * 8;
            }
            for (int p = j; p < kStagePad; p += S) {  // entries past the batch: read, never taken
                st.q[n + p] = make_longlong2(0, 0);
                st.e[n + p] = 0;
            }
            __syncwarp(gm);
            if (j < n) {  // every marked word belongs to some lane's site
                st.bm[wsite] = 0u;
                dup[wsite] = 0u;
            }
        }
        unsigned flagm = S > 1 ? __ballot_sync(gm, flag) >> gbase : 0u;  // the flagged steps

        // ---- serial phase: the group resolves the proposals in order ------------
        // accm: steps of the batch that accepted; done: those already written to
        // the lattice.  The lattice and the histogram are brought up to date in
        // parallel after the batch (and the lattice before an exact step).
        unsigned accm = 0, done = 0;
        const int Eb = Eo;
        uint32_t pcur = pbase + (uint32_t)Eo * 8u;
        int kk = 0;
        while (kk < n) {
            if (int_add) {
                if constexpr (S == 1) {
                    // ---- fast steps: integer decision and ln f step ---------------
                    // The step is computed speculatively; a step that needs more (a
                    // draw inside the bracket, a value with dropped bits, a binade
                    // crossing) leaves the loop before it changes anything.
                    const int En = Eo + dE;
                    const long long BF = lgf[En];  // beyond the window: kOutside
                    const long long D = BF - AF;
                    const bool acc = D < q1.x;
                    const bool unsure = (unsigned long long)D - (unsigned long long)q1.x < (unsigned long long)q1.y;
                    const long long cur = acc ? BF : AF;  // with dE = 0 both are the current shadow
                    const long long AF2 = cur + incF;
                    const uint32_t hc = (uint32_t)((unsigned long long)cur >> 32);
                    const uint32_t h2 = (uint32_t)((unsigned long long)AF2 >> 32);
                    if (!(unsure || (cur & 1) || (h2 ^ hc) > hc)) {
                        Eo = acc ? En : Eo;
                        AF = AF2;
                        lgf[Eo] = AF;
                        accm |= acc ? 1u : 0u;
                        kk = 1;
                    }
                } else {
                    // ---- step tree: lane j decides node j of the tree of the next DP
                    // steps (level lvl = the step, prefix pre = the decisions taken
                    // before it on the way there), all from the state at the start of
                    // the window; the ballots then follow the decisions from the
                    // root.  A node whose step needs more (a proposal whose
                    // neighbourhood may have changed, a draw inside the bracket, a
                    // value with dropped bits, a binade crossing) ends the window
                    // there, and the exact step below takes it.
                    //
                    // The path part of a window starting at step k0 needs no state.
                    struct Prep {
                        int m, oA, oB;
                        int e8[DP];  // energy changes of the window's steps (byte steps)
                        unsigned long long incA, incB;
                        longlong2 kq;
                    };
                    auto prep = [&](int k0) {
                        Prep P;
                        P.m = min(DP, n - k0);
                        int *e8l = P.e8;
#pragma unroll
                        for (int l = 0; l < DP; ++l) e8l[l] = st.e[k0 + l];
                        const int e8i = st.e[k0 + lvl];
                        P.kq = st.q[k0 + lvl];
                        // bins of the path to this node, as offsets from the current one
                        int post[DP > 1 ? DP - 1 : 1];
                        int oA = 0;
#pragma unroll
                        for (int l = 0; l < DP - 1; ++l) {
                            if (tb[l]) oA += e8l[l];
                            post[l] = oA;  // the bin after step l (l < lvl)
                        }
                        P.oA = oA;
                        P.oB = oA + e8i;
                        // ln f steps the path has already added to the two bins
                        int cA = 0, cB = 0;
#pragma unroll
                        for (int l = 0; l < DP - 1; ++l) {
                            if (tl[l]) {
                                cA += post[l] == P.oA ? 1 : 0;
                                cB += post[l] == P.oB ? 1 : 0;
                            }
                        }
                        P.incA = (unsigned long long)incF * (unsigned)cA;
                        P.incB = (unsigned long long)incF * (unsigned)cB;
                        return P;
                    };
                    for (;;) {
                        const Prep P = prep(kk);
                        const int m = P.m;
                        const longlong2 kq = P.kq;
                        // the node's decision (off the true path the values are
                        // meaningless, possibly wrapped, and never used)
                        const uint32_t pA = pcur + (uint32_t)P.oA, pB = pcur + (uint32_t)P.oB;
                        const long long Am = lds64(pA), Bm = lds64(pB);
                        const long long A = (long long)((unsigned long long)Am + P.incA);
                        const long long B = (long long)((unsigned long long)Bm + P.incB);
                        const long long D = (long long)((unsigned long long)B - (unsigned long long)A);
                        const bool dec = D < kq.x;
                        const bool unsure =
                            (unsigned long long)D - (unsigned long long)kq.x < (unsigned long long)kq.y;
                        const long long cur = dec ? B : A;
                        const long long A2 = (long long)((unsigned long long)cur + (unsigned long long)incF);
                        const uint32_t hc = (uint32_t)((unsigned long long)cur >> 32);
                        const uint32_t h2 = (uint32_t)((unsigned long long)A2 >> 32);
                        const bool act = lvl < m;
                        const bool bad = unsure || (cur & 1) || (h2 ^ hc) > hc;
                        const unsigned bd = __ballot_sync(gm, act && dec) >> gbase;
                        const unsigned bb = __ballot_sync(gm, act && bad) >> gbase;
                        // reached: every ancestor decided as the prefix says, and cleanly
                        const bool reached = act && (((bd ^ anc_bits) | bb) & anc_mask) == 0u;
                        const unsigned R = __ballot_sync(gm, reached) >> gbase;  // the true path
                        const int deep = 31 - __clz((int)R);
                        const bool dbad = (bb >> deep) & 1u;
                        const int c = (31 - __clz(deep + 1)) + (dbad ? 0 : 1);  // steps taken
                        const bool commit = reached && !bad;
                        // the decisions on the true path are the deepest node's prefix
                        const int bits = __shfl_sync(gm, (commit && dec) ? pre | (1 << lvl) : pre, deep, S);
                        // write the ln g values of the steps taken, level by level so
                        // that the latest value of a bin is the one that stays
                        const uint32_t pp = dec ? pB : pA;
#pragma unroll
                        for (int l = 0; l < DP; ++l) {
                            if (commit && lvl == l) sts64(pp, A2);
                            if (l + 1 < DP) __syncwarp(gm);
                        }
                        pcur = __shfl_sync(gm, (bad || !dec) ? pA : pB, deep, S);
                        AF = __shfl_sync(gm, bad ? A : A2, deep, S);
                        __syncwarp(gm);
                        accm |= ((unsigned)bits & ((1u << c) - 1u)) << kk;
                        kk += c;
                        if (c < m || kk >= n) break;
                    }
                }
                if constexpr (S > 1) Eo = (int)((pcur - pbase) >> 3);
                if (kk >= n) break;
            }
            if (S > 1 && int_add && ((flagm >> kk) & 1u)) {
                // ---- a proposal whose neighbourhood may have changed: its lane
                // recomputes it against the lattice as of this step, and the
                // windows go on from it
                if (((accm & ~done) >> j) & 1u) atomicXor(&lat[word], xr);
                done = accm;
                __syncwarp(gm);
                if (j == kk) {
                    const int c0 = spin_get<BITS>(lat, site);
                    const int nw0 = v + (v >= c0);
                    dE = energy_change<BITS>(lat, nb, c0, nw0);
                    xr = (uint32_t)(c0 ^ nw0) << ((site & (per - 1)) * BITS);
                    flag = false;
                    st.q[kk] = q1;
                    st.e[kk] = dE * 8;
                }
                flagm &= ~(1u << kk);
                __syncwarp(gm);
                continue;
            }
            // ---- the same step, every case done exactly ---------------------------
            if (S > 1) {  // the lattice as of this step
                if (((accm & ~done) >> j) & 1u) atomicXor(&lat[word], xr);
                done = accm;
                __syncwarp(gm);
            }
            const int ks = from_lane<S>(gm, site, kk);
            int kdE = from_lane<S>(gm, dE, kk);
            int kword = from_lane<S>(gm, word, kk);
            uint32_t kxr = from_lane<S>(gm, xr, kk);
            const long long tlo = from_lane<S>(gm, th.x, kk), thi = from_lane<S>(gm, th.y, kk);
            if (S > 1 && from_lane<S>(gm, (int)flag, kk)) {  // recompute against the current lattice
                const int kv = from_lane<S>(gm, v, kk);
                const int kc = spin_get<BITS>(lat, ks);
                const int knw = kv + (kv >= kc);
                kdE = energy_change<BITS>(lat, nbrs(ks, L, N, M.divL), kc, knw);
                kword = ks / per;
                kxr = (uint32_t)(kc ^ knw) << ((ks & (per - 1)) * BITS);
            }
            const int En = Eo + kdE;
            const long long BF = lgf[REWL_IDX(En, -kPad, M.B + kPad, tally.bad)];
            const long long D = BF - AF;
            bool acc = D < tlo;
            if (!acc && D < thi) {  // inside the bracket (never beyond the window)
                tally.slow += 1;
                const unsigned long long kU = from_lane<S>(gm, U, kk);
                const long long Ab = (AF & 1) ? lgb[REWL_IDX(Eo, 0, M.B, tally.bad)] : from_units(AF >> 1, ew);
                const long long Bb = (BF & 1) ? lgb[REWL_IDX(En, 0, M.B, tally.bad)] : from_units(BF >> 1, ew);
                acc = kdE == 0 ? true : exact_accept(Ab, Bb, kU, &tally.tie, t_io + (unsigned long long)kk);
            }
            const long long cur = acc ? BF : AF;
            const int Eb2 = acc ? En : Eo;
            long long AF2 = cur + incF;
            if (!int_add || (cur & 1)) {  // ln g(E) += ln f in binary64
                tally.seq += 1;
                const long long Ab = (cur & 1) ? lgb[REWL_IDX(Eb2, 0, M.B, tally.bad)] : from_units(cur >> 1, ew);
                const long long A2 = exact_add(Ab, lnf);
                lgb[REWL_IDX(Eb2, 0, M.B, tally.bad)] = A2;
                AF2 = shadow_of(A2, ew);
            } else {
                AF2 = round_shadow(AF2);
            }
            Eo = Eb2;
            AF = AF2;
            lgf[REWL_IDX(Eo, 0, M.B, tally.bad)] = AF;
            pcur = pbase + (uint32_t)Eo * 8u;
            if (acc) {
                if (S == 1 || j == 0) atomicXor(&lat[kword], kxr);
                accm |= 1u << kk;
            }
            done |= accm & (1u << kk);
            if (j == kk) dE = kdE;  // the lane's record of its step, for the histogram
            ++kk;
        }

        // ---- after the batch: lattice and histogram ----------------------------
        // (atomics whose result is not used: the walker does not wait for them)
        if (((accm & ~done) >> j) & 1u) atomicXor(&lat[word], xr);
        // the bin after step j: the batch's start plus the accepted moves up to j
        int x = (j < n && ((accm >> j) & 1u)) ? dE : 0;
#pragma unroll
        for (int o = 1; o < S; o <<= 1) {
            const int y = __shfl_up_sync(gm, x, o, S);
            if (j >= o) x += y;
        }
        const int bin = Eb + x;
        if (S == 1) {
            atomicAdd(&hg[REWL_IDX(bin, 0, M.B, tally.bad)], 1u);
        } else {  // one add per run of equal bins, by the run's last step
            const int nxt = __shfl_down_sync(gm, bin, 1, S);
            const bool last = j < n && (j == n - 1 || nxt != bin);
            const unsigned ends = __ballot_sync(gm, last) >> gbase;
            const unsigned below = ends & ((1u << j) - 1u);  // j < 32
            if (last) atomicAdd(&hg[REWL_IDX(bin, 0, M.B, tally.bad)], (uint32_t)(j - (below ? 31 - __clz((int)below) : -1)));
        }
        nacc += (uint32_t)__popc(accm);
        if (S > 1) __syncwarp(gm);
        t_io += (unsigned long long)n;
    }
    if (S > 1) __syncwarp(gm);
    // the binary64 array from the authoritative shadow
    for (int b = j; b < M.B; b += S) {
        const long long F = lgf[b];
        if (!(F & 1)) lgb[b] = from_units(F >> 1, ew);
    }
    tally.acc += nacc;
    E_io = Eo + lo;
}

// P walkers g0 .. g0 + P - 1 of one instance: stage their lattices in shared
// memory (LG = false; LG = true keeps large lattices in global memory), run K
// steps (one lane group per walker), write the lattices back.  The binary64
// ln g and the histogram of each walker stay in global memory: the launch
// reads ln g once to build the shadow and writes it back once at the end.
template <int BITS, int S, bool LG>
__device__ void sweep_block(const Model &M, const State &Sg, int g0, int P, const Layout &lay, unsigned char *smem) {
    if (*(volatile unsigned int *)&Sg.ctl->all_done) return;
    const int nbw = (min(M.N, kMarkBits) + 31) / 32;  // conflict-mark words
    for (int p = 0; p < P; ++p) {
        const int g = g0 + p;
        if (g >= M.G || Sg.done[g / M.m]) continue;
        unsigned char *base = smem + (size_t)p * lay.stride;
        if (!LG) {
            uint32_t *lat = reinterpret_cast<uint32_t *>(base + lay.off_lat);
            const uint32_t *src_lat = Sg.spins + (size_t)Sg.slot_cfg[g] * M.wpc;
            for (int i = threadIdx.x; i < M.wpc; i += blockDim.x) lat[i] = src_lat[i];
        }
        if (S > 1) {
            uint32_t *bm = reinterpret_cast<uint32_t *>(base + lay.off_bm);
            for (int i = threadIdx.x; i < 2 * nbw; i += blockDim.x) bm[i] = 0u;
        }
    }
    __syncthreads();

    const int grp = threadIdx.x / S, g = g0 + grp;
    Tally tally{};
    if (grp < P && g < M.G && !Sg.done[g / M.m]) {
        unsigned char *base = smem + (size_t)grp * lay.stride;
        Stage st;
        st.q = reinterpret_cast<longlong2 *>(base + lay.off_q);
        st.e = reinterpret_cast<int *>(base + lay.off_e);
        st.bm = reinterpret_cast<uint32_t *>(base + lay.off_bm);
        st.nbw = nbw;
        st.mmask = M.N > kMarkBits ? (uint32_t)(kMarkBits - 1) : 0xffffffffu;
        const int w = g / M.m;
        const uint32_t c = Sg.slot_cfg[g];
        int E = Sg.cfg_E[c];
        unsigned long long t = Sg.t[g];
        uint32_t *lat = LG ? Sg.spins + (size_t)c * M.wpc : reinterpret_cast<uint32_t *>(base + lay.off_lat);
        // one lane with global lattices: the shadow is in global memory too
        long long *lgf = (S == 1 && LG) ? Sg.shadow + (size_t)g * (M.B + 2 * kPad) + kPad
                                        : reinterpret_cast<long long *>(base + lay.off_lgf) + kPad;
        walker_sweep<BITS, S>(M, lat, reinterpret_cast<long long *>(Sg.lng + (size_t)g * M.B), lgf,
                              Sg.H + (size_t)g * M.B, st, g, Sg.e_lo[w], Sg.lnf[w], E, t, tally);
        if ((threadIdx.x & (S - 1)) == 0) {
            Sg.cfg_E[c] = E;
            Sg.t[g] = t;
            atomicAdd(&Sg.ctl->flips, (unsigned long long)M.K);
            atomicAdd(&Sg.ctl->accepted, (unsigned long long)tally.acc);
            if (tally.slow) atomicAdd(&Sg.ctl->slow, tally.slow);
            flush_ties(Sg, g, tally.tie);
            if (tally.seq) atomicAdd(&Sg.ctl->seq, (unsigned long long)tally.seq);
#ifdef REWL_DEBUG_CHECKS
            if (tally.bad) atomicOr(&Sg.ctl->error, ERR_BOUNDS);
#endif
        }
    }
    __syncthreads();

    if (!LG) {
        for (int p = 0; p < P; ++p) {
            const int gg = g0 + p;
            if (gg >= M.G || Sg.done[gg / M.m]) continue;
            const uint32_t *lat = reinterpret_cast<const uint32_t *>(smem + (size_t)p * lay.stride + lay.off_lat);
            uint32_t *dst_lat = Sg.spins + (size_t)Sg.slot_cfg[gg] * M.wpc;
            for (int i = threadIdx.x; i < M.wpc; i += blockDim.x) dst_lat[i] = lat[i];
        }
    }
}

template <int BITS, int S, bool LG>
__global__ void __launch_bounds__(256) sweep_fast_kernel(Model M, State Sg, int P, Layout lay) {
    extern __shared__ __align__(16) unsigned char smem[];
    sweep_block<BITS, S, LG>(M, Sg, blockIdx.x * P, P, lay, smem);
}

// Persistent batched sweep: each CTA takes the next item from *queue.
template <int BITS, int S>
__global__ void __launch_bounds__(256) batch_sweep_kernel(const InstDev *inst, const SweepItem *items, int n_items,
                                                          unsigned int *queue) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int next;
    for (;;) {
        if (threadIdx.x == 0) next = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int i = next;
        if (i >= n_items) break;
        const SweepItem it = items[i];
        const Model M = inst[it.inst].M;
        const State Sg = inst[it.inst].S;
        const Layout lay = inst[it.inst].lay;
        sweep_block<BITS, S, false>(M, Sg, it.g0, it.P, lay, smem);
        __syncthreads();
    }
}

// Batched one-lane sweep with every walker's state in global memory: thread i
// runs walker items[i] (any instance of this spin packing) for K steps.
template <int BITS>
__global__ void __launch_bounds__(256) batch_walker_kernel(const InstDev *inst, const WalkerItem *items, int n_items) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_items) return;
    const WalkerItem it = items[i];
    const Model &M = inst[it.inst].M;
    const State &Sg = inst[it.inst].S;
    if (*(volatile unsigned int *)&Sg.ctl->all_done) return;
    const int g = it.g;
    if (Sg.done[g / M.m]) return;
    const Model Mr = M;
    const State Sr = Sg;
    Stage st{};
    Tally tally{};
    const int w = g / Mr.m;
    const uint32_t c = Sr.slot_cfg[g];
    int E = Sr.cfg_E[c];
    unsigned long long t = Sr.t[g];
    walker_sweep<BITS, 1>(Mr, Sr.spins + (size_t)c * Mr.wpc, reinterpret_cast<long long *>(Sr.lng + (size_t)g * Mr.B),
                          Sr.shadow + (size_t)g * (Mr.B + 2 * kPad) + kPad, Sr.H + (size_t)g * Mr.B, st, g, Sr.e_lo[w],
                          Sr.lnf[w], E, t, tally);
    Sr.cfg_E[c] = E;
    Sr.t[g] = t;
    atomicAdd(&Sr.ctl->flips, (unsigned long long)Mr.K);
    atomicAdd(&Sr.ctl->accepted, (unsigned long long)tally.acc);
    if (tally.slow) atomicAdd(&Sr.ctl->slow, tally.slow);
    flush_ties(Sr, g, tally.tie);
    if (tally.seq) atomicAdd(&Sr.ctl->seq, (unsigned long long)tally.seq);
#ifdef REWL_DEBUG_CHECKS
    if (tally.bad) atomicOr(&Sr.ctl->error, ERR_BOUNDS);
#endif
}

Layout make_layout(const Model &M, int S, bool lat_global) {
    auto al = [](int x) { return (x + 15) & ~15; };
    Layout l{};
    int off = 0;
    if (S == 1 && lat_global) {  // every part of the walker's state in global memory
        l.off_lgf = l.off_lat = l.off_q = l.off_e = l.off_bm = -1;
        l.stride = 0;
        return l;
    }
    l.off_lgf = off;
    off += al((M.B + 2 * kPad) * 8);
    l.off_lat = -1;
    if (!lat_global) {
        l.off_lat = off;
        off += al(M.wpc * 4);
    }
    if (S > 1) {  // entries past the batch: the step tree reads up to six ahead
        l.off_q = off;
        off += al((S + kStagePad) * 16);
        l.off_e = off;
        off += al((S + kStagePad) * 4);
        l.off_bm = off;
        off += al(2 * ((min(M.N, kMarkBits) + 31) / 32) * 4);
    }
    l.stride = al(off);
    return l;
}

template <int BITS, int S, bool LG>
cudaError_t launch_lg(const Model &M, const State &St, const SweepPlan &p, cudaStream_t s, bool prepare) {
    const Layout lay = make_layout(M, S, LG);
    if (prepare)
        return cudaFuncSetAttribute(sweep_fast_kernel<BITS, S, LG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)p.smem);
    sweep_fast_kernel<BITS, S, LG><<<p.grid, p.threads, p.smem, s>>>(M, St, p.P, lay);
    return cudaGetLastError();
}

template <int BITS, int S>
cudaError_t launch_t(const Model &M, const State &St, const SweepPlan &p, cudaStream_t s, bool prepare) {
    return p.lat_global ? launch_lg<BITS, S, true>(M, St, p, s, prepare)
                        : launch_lg<BITS, S, false>(M, St, p, s, prepare);
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

size_t fast_smem_per_walker(const Model &M, int lanes, bool lat_global) {
    return (size_t)fast::make_layout(M, lanes, lat_global).stride;
}

Layout fast_layout(const Model &M, int lanes, bool lat_global) { return fast::make_layout(M, lanes, lat_global); }

namespace {
template <int BITS, int S>
cudaError_t batch_launch_t(const InstDev *inst, const SweepItem *items, int n_items, unsigned int *queue, int grid,
                           int threads, size_t smem, cudaStream_t s, bool prepare) {
    if (prepare)
        return cudaFuncSetAttribute(fast::batch_sweep_kernel<BITS, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    if (n_items <= 0) return cudaSuccess;
    fast::batch_sweep_kernel<BITS, S><<<grid, threads, smem, s>>>(inst, items, n_items, queue);
    return cudaGetLastError();
}
template <int BITS>
cudaError_t batch_dispatch(int lanes, const InstDev *inst, const SweepItem *items, int n_items, unsigned int *queue,
                           int grid, int threads, size_t smem, cudaStream_t s, bool prepare) {
    switch (lanes) {
    case 1: return batch_launch_t<BITS, 1>(inst, items, n_items, queue, grid, threads, smem, s, prepare);
    case 2: return batch_launch_t<BITS, 2>(inst, items, n_items, queue, grid, threads, smem, s, prepare);
    case 4: return batch_launch_t<BITS, 4>(inst, items, n_items, queue, grid, threads, smem, s, prepare);
    case 8: return batch_launch_t<BITS, 8>(inst, items, n_items, queue, grid, threads, smem, s, prepare);
    case 16: return batch_launch_t<BITS, 16>(inst, items, n_items, queue, grid, threads, smem, s, prepare);
    default: return batch_launch_t<BITS, 32>(inst, items, n_items, queue, grid, threads, smem, s, prepare);
    }
}
template <int BITS, int S>
int occupancy_t(int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fast::batch_sweep_kernel<BITS, S>, threads, smem) !=
        cudaSuccess)
        return 0;
    return n;
}
}  // namespace

cudaError_t launch_batch_sweep(int bits, int lanes, const InstDev *inst, const SweepItem *items, int n_items,
                               unsigned int *queue, int grid, int threads, size_t smem, cudaStream_t s,
                               bool prepare) {
    return bits == 8 ? batch_dispatch<8>(lanes, inst, items, n_items, queue, grid, threads, smem, s, prepare)
                     : batch_dispatch<4>(lanes, inst, items, n_items, queue, grid, threads, smem, s, prepare);
}

int batch_sweep_ctas_per_sm(int bits, int lanes, int threads, size_t smem) {
    if (bits == 8) {
        switch (lanes) {
        case 1: return occupancy_t<8, 1>(threads, smem);
        case 2: return occupancy_t<8, 2>(threads, smem);
        case 4: return occupancy_t<8, 4>(threads, smem);
        case 8: return occupancy_t<8, 8>(threads, smem);
        case 16: return occupancy_t<8, 16>(threads, smem);
        default: return occupancy_t<8, 32>(threads, smem);
        }
    }
    switch (lanes) {
    case 1: return occupancy_t<4, 1>(threads, smem);
    case 2: return occupancy_t<4, 2>(threads, smem);
    case 4: return occupancy_t<4, 4>(threads, smem);
    case 8: return occupancy_t<4, 8>(threads, smem);
    case 16: return occupancy_t<4, 16>(threads, smem);
    default: return occupancy_t<4, 32>(threads, smem);
    }
}

cudaError_t launch_batch_walkers(int bits, const InstDev *inst, const WalkerItem *items, int n_items, int grid,
                                 int threads, cudaStream_t s, bool prepare) {
    if (prepare) return cudaSuccess;
    if (n_items <= 0) return cudaSuccess;
    if (bits == 8) fast::batch_walker_kernel<8><<<grid, threads, 0, s>>>(inst, items, n_items);
    else fast::batch_walker_kernel<4><<<grid, threads, 0, s>>>(inst, items, n_items);
    return cudaGetLastError();
}

int batch_walkers_ctas_per_sm(int bits, int threads) {
    int n = 0;
    cudaError_t e = bits == 8 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fast::batch_walker_kernel<8>, threads, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fast::batch_walker_kernel<4>, threads, 0);
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_sweep_fast(const Model &M, const State &S, const SweepPlan &p, cudaStream_t s, bool prepare) {
    return M.bits == 8 ? fast::dispatch_s<8>(M, S, p, s, prepare) : fast::dispatch_s<4>(M, S, p, s, prepare);
}

}  // namespace rewl
