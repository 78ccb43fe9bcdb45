// The lock-free reduction of the residual columns (included by cr_h1.cu,
// once per instance, inside a namespace that defines ICAP, TT and
// RED_BLOCKS; deliberately without an include guard).
static_assert(TT % 32 == 0 && ICAP % 32 == 0 && ICAP >= 128, "warp-sized tiles and inbox");

struct WarpSmem {
    uint64_t f[2][FCAP];   // the front: sorted, distinct (double buffered)
    uint64_t in[ICAP];     // the inbox: unsorted, repeated entries cancel in pairs
    uint64_t c[DMAX + 1];  // a staged published column
    uint64_t cand[128];    // candidates of a front refill
    uint64_t ta[TT + 1];   // merge windows
    uint64_t tb[TT + 1];
    int q[DMAX];           // merge scratch
    int pc[DMAX + 1];
};
constexpr size_t RED_SMEM = RED_WARPS * sizeof(WarpSmem);

__device__ __forceinline__ int warp_excl_scan(int x, int &total) {
    const int lane = threadIdx.x & 31;
    int incl = x;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    return incl - x;
}

// out = A xor D with D sorted in shared memory; A in global memory (read
// through L2, AG = true) or in shared memory.  One pass over A: the insertion
// points of D are found by binary search, then A is streamed in chunks of
// 256 with each entry shifted by the insertions and cancellations before it.
template <bool AG>
__device__ __forceinline__ uint64_t ld_a(const uint64_t *A, int i) {
    return AG ? ld_cg(A + i) : A[i];
}

template <bool AG>
__device__ int insert_merge(const uint64_t *A, int na, const uint64_t *D, int nD, uint64_t *out, WarpSmem &sm) {
    const int lane = threadIdx.x & 31;
    // 1. insertion positions of D in A and cancellations
    for (int k = lane; k < nD; k += 32) {
        uint64_t x = D[k];
        int lo = 0, hi = na;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (ld_a<AG>(A, mid) < x) lo = mid + 1; else hi = mid;
        }
        sm.q[k] = lo;
        sm.pc[k + 1] = (lo < na && ld_a<AG>(A, lo) == x) ? 1 : 0;
    }
    __syncwarp();
    // 2. exclusive prefix counts of cancellations: pc[k] = cancelled among D[0..k)
    int run = 0;
    for (int base = 0; base < nD; base += 32) {
        int k = base + lane;
        int f = k < nD ? sm.pc[k + 1] : 0;
        int tot;
        int ex = warp_excl_scan(f, tot);
        __syncwarp();
        if (k < nD) sm.pc[k] = run + ex;
        run += tot;
        __syncwarp();
    }
    if (lane == 0) sm.pc[nD] = run;
    __syncwarp();
    const int cancelled = run;
    // 3. the surviving entries of D
    for (int k = lane; k < nD; k += 32) {
        bool eq = sm.pc[k + 1] - sm.pc[k];
        if (!eq) out[sm.q[k] + k - 2 * sm.pc[k]] = D[k];
    }
    // 4. stream A
    for (int c0 = 0; c0 < na; c0 += 256) {
        // insertion points that fall into this chunk: q in [c0, c0 + 256)
        int lo = 0, hi = nD;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (sm.q[mid] < c0) lo = mid + 1; else hi = mid;
        }
        const int klo = lo;
        hi = nD;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (sm.q[mid] < c0 + 256) lo = mid + 1; else hi = mid;
        }
        const int khi = lo;
        uint64_t v[8];
#pragma unroll
        for (int t = 0; t < 8; t++) {
            int i = c0 + lane + 32 * t;
            v[t] = i < na ? ld_a<AG>(A, i) : 0;
        }
        int kk = klo;  // #{k : q[k] <= i}, carried forward: i grows with t
#pragma unroll
        for (int t = 0; t < 8; t++) {
            int i = c0 + lane + 32 * t;
            if (i >= na) break;
            while (kk < khi && sm.q[kk] <= i) kk++;
            bool cancel = kk > 0 && sm.q[kk - 1] == i && (sm.pc[kk] - sm.pc[kk - 1]);
            if (!cancel) out[i + kk - 2 * sm.pc[kk]] = v[t];
        }
    }
    __syncwarp();
    return na + nD - 2 * cancelled;
}

// out = A xor B for sorted, distinct runs A and B, each read from global
// memory through L2 (AG / BG) or from shared memory.  The merged order is
// produced in tiles of TT positions: both runs are staged in windows of TT+1
// entries (coalesced loads; the first TT+1 merged entries lie in them), each
// lane merges TT/32 positions found by a merge-path search in shared memory,
// and an entry equal to its neighbour in the merged order cancels.  Returns
// the length of out, or -1 if it would exceed cap.
template <bool AG, bool BG>
__device__ int tiled_xor(const uint64_t *A, int na, const uint64_t *B, int nb, uint64_t *out, int cap, WarpSmem &sm) {
    constexpr int PER = TT / 32;
    const int lane = threadIdx.x & 31;
    uint64_t *ta = sm.ta, *tb = sm.tb;
    int i = 0, j = 0, no = 0;
    uint64_t prev = 0;
    bool hasprev = false;
    while (i + j < na + nb) {
#pragma unroll
        for (int k = lane; k <= TT; k += 32) {
            ta[k] = i + k < na ? (AG ? ld_cg(A + i + k) : A[i + k]) : ~0ull;
            tb[k] = j + k < nb ? (BG ? ld_cg(B + j + k) : B[j + k]) : ~0ull;
        }
        __syncwarp();
        const int left = na + nb - i - j;
        const int T = min(TT, left);
        const int wa = min(TT + 1, na - i), wb = min(TT + 1, nb - j);
        const int s = min(lane * PER, T), e = min(s + PER, T);
        // A entries among the first d merged positions (ties: A first), for d =
        // this lane's start s and the tile's end T: two binary searches run in step
        int ia, ca;
        {
            int lo1 = max(0, s - wb), hi1 = min(s, wa), lo2 = max(0, T - wb), hi2 = min(T, wa);
            while (lo1 < hi1 || lo2 < hi2) {
                const int m1 = (lo1 + hi1) >> 1, m2 = (lo2 + hi2) >> 1;
                const bool g1 = lo1 < hi1, g2 = lo2 < hi2;
                const uint64_t a1 = g1 ? ta[m1] : 0ull, b1 = g1 ? tb[s - 1 - m1] : 0ull;
                const uint64_t a2 = g2 ? ta[m2] : 0ull, b2 = g2 ? tb[T - 1 - m2] : 0ull;
                if (g1) { if (a1 <= b1) lo1 = m1 + 1; else hi1 = m1; }
                if (g2) { if (a2 <= b2) lo2 = m2 + 1; else hi2 = m2; }
            }
            ia = lo1;
            ca = lo2;
        }
        int ib = s - ia;
        const uint64_t la = ca > 0 ? ta[ca - 1] : 0ull, lb = T - ca > 0 ? tb[T - ca - 1] : 0ull;
        uint64_t pv = prev;
        bool hp = hasprev;
        if (s > 0) {
            const uint64_t pa = ia > 0 ? ta[ia - 1] : 0ull, pb = ib > 0 ? tb[ib - 1] : 0ull;
            pv = pa > pb ? pa : pb;
            hp = true;
        }
        auto take = [&]() {
            if (ia < wa && (ib >= wb || ta[ia] <= tb[ib])) return ta[ia++];
            return tb[ib++];
        };
        uint64_t cur = s < e ? take() : 0ull;
        uint64_t kv[PER];
        unsigned kf = 0;
#pragma unroll
        for (int t = 0; t < PER; t++) {
            kv[t] = 0ull;
            if (s + t < e) {
                const bool hn = s + t + 1 < left;
                const uint64_t nx = hn ? take() : 0ull;  // the successor (may lie past the tile)
                const bool dup = (hp && pv == cur) || (hn && nx == cur);
                kv[t] = cur;
                if (!dup) kf |= 1u << t;
                pv = cur;
                hp = true;
                cur = nx;
            }
        }
        int total;
        const int base = warp_excl_scan(__popc(kf), total);
        if (no + total > cap) return -1;
#pragma unroll
        for (int t = 0; t < PER; t++)
            if ((kf >> t) & 1u) out[no + base + __popc(kf & ((1u << t) - 1u))] = kv[t];
        no += total;
        prev = la > lb ? la : lb;
        hasprev = true;
        i += ca;
        j += T - ca;
        __syncwarp();
    }
    return no;
}

// base <- base[start..nb) xor mid[mstart..nm); the middle level becomes empty
__device__ bool merge_mid(const RedParams &R, Work &W, WarpSmem &sm, RedStats &st) {
    int nmid = W.nm - W.mstart;
    if (nmid == 0) return true;
    int na = W.nb - W.start;
    const uint64_t *A = W.g[W.bown] + W.start;
    if ((int64_t)na + nmid > W.cap && !grow_to(R, W, (int64_t)na + nmid)) return false;
    int x = W.bown ^ 1;
    int n = tiled_xor<true, true>(A, na, W.mg[W.mown] + W.mstart, nmid, W.g[x], W.cap, sm);
    __threadfence_block();
    if (n < 0) return false;
    W.bown = x;
    W.nb = n;
    W.start = 0;
    W.nm = W.mstart = 0;
    st.merged += (unsigned long long)(na + nmid);
    return true;
}

// ascending sort of a[0..n) in shared memory by the warp; n a power of two, 2 <= n <= 1024.
// The compare-exchanges of one stage touch disjoint pairs, so a lane loads
// four pairs before it writes any: the sort runs on a lone warp at the end of
// the reduction, where dependent shared-memory round trips set its time.
__device__ void warp_bitonic(uint64_t *a, int n) {
    const int lane = threadIdx.x & 31;
    const int half = n >> 1;
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t0 = lane; t0 < half; t0 += 4 * 32) {
                int i[4];
                uint64_t x[4], y[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int t = t0 + 32 * u;
                    i[u] = ((t & ~(j - 1)) << 1) | (t & (j - 1));  // t with a zero bit inserted at j
                    x[u] = t < half ? a[i[u]] : 0ull;
                    y[u] = t < half ? a[i[u] | j] : 0ull;
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    if (t0 + 32 * u < half && (x[u] > y[u]) == ((i[u] & k) == 0)) {
                        a[i[u]] = y[u];
                        a[i[u] | j] = x[u];
                    }
                }
            }
            __syncwarp();
        }
    }
}

// sort the inbox and cancel repeated entries in pairs: in[0..n) becomes
// sorted and distinct; returns n.  Survivors (the first entry of a run of odd
// length) are marked in a read-only pass, then compacted in place chunk by
// chunk (a chunk's survivors land no further than its own slots).
__device__ int sort_inbox(WarpSmem &sm, int ni) {
    const int lane = threadIdx.x & 31;
    if (ni == 0) return 0;
    int n2 = 32;
    while (n2 < ni) n2 <<= 1;
    for (int i = ni + lane; i < n2; i += 32) sm.in[i] = ~0ull;
    __syncwarp();
    warp_bitonic(sm.in, n2);
    unsigned keep = 0;  // bit t: entry t*32 + lane survives
#pragma unroll 4
    for (int t = 0; t * 32 < n2; t++) {
        const int i = t * 32 + lane;
        const uint64_t v = sm.in[i];
        if (v != ~0ull && (i == 0 || sm.in[i - 1] != v)) {
            int r = 1;
            while (i + r < n2 && sm.in[i + r] == v) r++;
            if (r & 1) keep |= 1u << t;
        }
    }
    __syncwarp();
    // compaction four chunks at a time: a chunk's survivors land no further
    // than its own slots, so the chunks read ahead are not yet overwritten
    const unsigned lt = (1u << lane) - 1u;
    int n = 0;
    for (int t0 = 0; t0 * 32 < n2; t0 += 4) {
        uint64_t v[4];
        unsigned m[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int t = t0 + u;
            const bool in = t * 32 < n2;
            v[u] = in ? sm.in[t * 32 + lane] : 0ull;
            m[u] = __ballot_sync(0xFFFFFFFFu, in && ((keep >> t) & 1u));
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if ((m[u] >> lane) & 1u) sm.in[n + __popc(m[u] & lt)] = v[u];
            n += __popc(m[u]);
        }
        __syncwarp();
    }
    return n;
}

// fold the inbox into the middle level (long columns) or into the base
__device__ bool flush_inbox(const RedParams &R, Work &W, WarpSmem &sm, RedStats &st) {
    TMARK(tf);
    const int n = sort_inbox(sm, W.ni);
    W.ni = 0;
    if (n == 0) return true;
    if (!W.mid_on && W.nb - W.start > MID_ON) {
        if (!W.mg[0]) {
            const int lane = threadIdx.x & 31;
            unsigned long long off = 0;
            if (lane == 0) off = atomicAdd(R.pool_top, (unsigned long long)(2 * MIDCAP));
            off = __shfl_sync(0xFFFFFFFFu, off, 0);
            if ((int64_t)(off + 2 * MIDCAP) > R.pool_cap) return false;
            W.mg[0] = R.pool + off;
            W.mg[1] = R.pool + off + MIDCAP;
        }
        W.mid_on = true;
        W.mown = 0;
        W.nm = W.mstart = 0;
    }
    if (W.mid_on) {
        const int nmid = W.nm - W.mstart, x = W.mown ^ 1;
        const int m = tiled_xor<true, false>(W.mg[W.mown] + W.mstart, nmid, sm.in, n, W.mg[x], MIDCAP, sm);
        __threadfence_block();
        if (m < 0) return false;
        W.mown = x;
        W.nm = m;
        W.mstart = 0;
        st.merged += (unsigned long long)(nmid + n);
        if (W.nm > MIDMAX && !merge_mid(R, W, sm, st)) return false;
    } else {
        const int na = W.nb - W.start;
        const uint64_t *A = W.g[W.bown] + W.start;
        if ((int64_t)na + n > W.cap && !grow_to(R, W, (int64_t)na + n)) return false;
        const int x = W.bown ^ 1;
        const int m = tiled_xor<true, false>(A, na, sm.in, n, W.g[x], W.cap, sm);
        __threadfence_block();
        if (m < 0) return false;
        W.bown = x;
        W.nb = m;
        W.start = 0;
        st.merged += (unsigned long long)(na + n);
    }
    st.flush++;
    TADD(st, 5, tf);
    return true;
}

// append x (lane e < m holds one entry) to the inbox
__device__ __forceinline__ bool inbox_add(const RedParams &R, Work &W, WarpSmem &sm, uint64_t x, int m,
                                          RedStats &st) {
    const int lane = threadIdx.x & 31;
    if (W.ni + m > ICAP && !flush_inbox(R, W, sm, st)) return false;
    if (lane < m) sm.in[W.ni + lane] = x;
    W.ni += m;
    __syncwarp();
    return true;
}

// move the front's entries above t to the inbox; tau becomes t
__device__ bool lower_tau(const RedParams &R, Work &W, WarpSmem &sm, uint64_t t, RedStats &st) {
    const int lane = threadIdx.x & 31;
    int lo = W.fh, hi = W.fn;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sm.f[W.fb][mid] <= t) lo = mid + 1; else hi = mid;
    }
    for (int s = lo; s < W.fn; s += 32) {
        const int m = min(32, W.fn - s);
        const uint64_t x = lane < m ? sm.f[W.fb][s + lane] : 0ull;
        if (!inbox_add(R, W, sm, x, m, st)) return false;
    }
    W.fn = lo;
    W.tau = t;
    return true;
}

// The front is empty: take every entry of inbox xor middle xor base up to a
// cut.  The cut is the smaller of the 32nd remaining entries of base and
// middle, so that their entries up to it are in one 32-entry window each;
// the candidates are sorted and entries present an even number of times cancel.
__device__ bool front_refill(const RedParams &R, Work &W, WarpSmem &sm, RedStats &st) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    while (W.tau != ~0ull) {
        const int nbr = W.nb - W.start, nmr = W.mid_on ? W.nm - W.mstart : 0;
        const uint64_t bv = lane < nbr ? ld_cg(W.g[W.bown] + W.start + lane) : ~0ull;
        const uint64_t mv = lane < nmr ? ld_cg(W.mg[W.mown] + W.mstart + lane) : ~0ull;
        const uint64_t cb = __shfl_sync(0xFFFFFFFFu, bv, 31), cm = __shfl_sync(0xFFFFFFFFu, mv, 31);
        uint64_t cut = nbr > 32 ? cb : ~0ull;
        if (nmr > 32 && cm < cut) cut = cm;
        int nic = 0;
#pragma unroll 4
        for (int i0 = 0; i0 < W.ni; i0 += 32) {
            const int i = i0 + lane;
            nic += __popc(__ballot_sync(0xFFFFFFFFu, i < W.ni && sm.in[i] <= cut));
        }
        if (nic > 64) {  // the inbox joins the sorted levels first
            if (!flush_inbox(R, W, sm, st)) return false;
            continue;
        }
        const bool tb = lane < nbr && bv <= cut, tm = lane < nmr && mv <= cut;
        sm.cand[lane] = tb ? bv : ~0ull;
        sm.cand[32 + lane] = tm ? mv : ~0ull;
        sm.cand[64 + lane] = ~0ull;
        sm.cand[96 + lane] = ~0ull;
        __syncwarp();
        // four chunks read before any is written: kept entries land no further
        // than their own chunk's slots, so the chunks read ahead are intact
        int nk = 0, nt = 0;
        for (int i0 = 0; i0 < W.ni; i0 += 4 * 32) {
            uint64_t x[4];
            unsigned mt[4], mk[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int i = i0 + 32 * u + lane;
                const bool valid = i < W.ni;
                x[u] = valid ? sm.in[i] : ~0ull;
                const bool take = valid && x[u] <= cut;
                mt[u] = __ballot_sync(0xFFFFFFFFu, take);
                mk[u] = __ballot_sync(0xFFFFFFFFu, valid && !take);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if ((mt[u] >> lane) & 1u) sm.cand[64 + nk + __popc(mt[u] & lt)] = x[u];
                if ((mk[u] >> lane) & 1u) sm.in[nt + __popc(mk[u] & lt)] = x[u];
                nk += __popc(mt[u]);
                nt += __popc(mk[u]);
            }
            __syncwarp();
        }
        W.ni = nt;
        W.start += __popc(__ballot_sync(0xFFFFFFFFu, tb));
        if (W.mid_on) W.mstart += __popc(__ballot_sync(0xFFFFFFFFu, tm));
        warp_bitonic(sm.cand, 128);
        uint64_t *out = sm.f[W.fb];
        int ns = 0;
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const int i = t * 32 + lane;
            const uint64_t v = sm.cand[i];
            bool keep = false;
            if (v != ~0ull && (i == 0 || sm.cand[i - 1] != v)) {
                int r = 1;
                while (i + r < 128 && sm.cand[i + r] == v) r++;
                keep = r & 1;
            }
            const unsigned m = __ballot_sync(0xFFFFFFFFu, keep);
            if (keep) out[ns + __popc(m & lt)] = v;
            ns += __popc(m);
        }
        __syncwarp();
        W.fh = 0;
        W.fn = ns;
        W.tau = cut;
        if (ns > 0) return true;
    }
    return true;
}

// the working column's pivot after a refill of an empty front; ~0 if the column is empty
__device__ __forceinline__ bool front_ready(const RedParams &R, Work &W, WarpSmem &sm, RedStats &st) {
    if (W.fh < W.fn) return true;
    TMARK(tr);
    const bool ok = front_refill(R, W, sm, st);
    TADD(st, 0, tr);
    return ok;
}

// Toggle x1 < x2 < x3 (the first m of them; all above the removed pivot).
// Entries up to tau are merged into the front, the rest go to the inbox.
// Added tails usually land among the front's first entries, so the merge is
// done in place when every entry to toggle falls among the first 32 and the
// front has room at its head: the entries before the last toggled position
// shift by the net count of insertions and cancellations behind them, the
// rest stay where they are.  Otherwise one pass writes the merged front into
// the other buffer, leaving FRONT_SLACK free slots at its head.
constexpr int FRONT_SLACK = 4;
__device__ bool toggle_small(const RedParams &R, Work &W, WarpSmem &sm, uint64_t x1, uint64_t x2, uint64_t x3,
                             int m, RedStats &st) {
    const int lane = threadIdx.x & 31;
    int mlo = (m > 0 && x1 <= W.tau) + (m > 1 && x2 <= W.tau) + (m > 2 && x3 <= W.tau);
    if (mlo > 0 && W.fn - W.fh + mlo > FCAP) {
        if (!lower_tau(R, W, sm, sm.f[W.fb][W.fh + FCAP / 2 - 1], st)) return false;
        mlo = (m > 0 && x1 <= W.tau) + (m > 1 && x2 <= W.tau) + (m > 2 && x3 <= W.tau);
    }
    const int mhi = m - mlo;
    if (mhi > 0) {
        const int e = mlo + lane;
        const uint64_t v = e == 0 ? x1 : (e == 1 ? x2 : x3);
        if (!inbox_add(R, W, sm, v, mhi, st)) return false;
    }
    if (mlo == 0) return true;
    const int nd = W.fn - W.fh;
    const uint64_t v0 = x1, v1 = mlo > 1 ? x2 : ~0ull, v2 = mlo > 2 ? x3 : ~0ull;
    {
        // in place: lane i holds the front's entry i (i < 32)
        uint64_t *F = &sm.f[W.fb][W.fh];
        const bool live = lane < nd;
        const uint64_t d = live ? F[lane] : ~0ull;
        const unsigned lt0 = __ballot_sync(0xFFFFFFFFu, live && d < v0), eq0m = __ballot_sync(0xFFFFFFFFu, live && d == v0);
        const unsigned lt1 = __ballot_sync(0xFFFFFFFFu, live && d < v1), eq1m = __ballot_sync(0xFFFFFFFFu, live && d == v1);
        const unsigned lt2 = __ballot_sync(0xFFFFFFFFu, live && d < v2), eq2m = __ballot_sync(0xFFFFFFFFu, live && d == v2);
        const int q0 = __popc(lt0), q1 = __popc(lt1), q2 = __popc(lt2);
        const int e0 = eq0m != 0, e1 = mlo > 1 && eq1m != 0, e2 = mlo > 2 && eq2m != 0;
        const int E = e0 + e1 + e2;
        const int qmax = mlo > 2 ? q2 : (mlo > 1 ? q1 : q0);  // the last toggled position
        const int shift = mlo - 2 * E;                        // net entries added
        if ((nd <= 32 || qmax < 32) && W.fh >= shift) {
            // entry i moves by (insertions before it) - (cancellations before it) - shift
            const int ins = (v0 < d && !e0) + (mlo > 1 && v1 < d && !e1) + (mlo > 2 && v2 < d && !e2);
            const int can = (v0 < d && e0) + (mlo > 1 && v1 < d && e1) + (mlo > 2 && v2 < d && e2);
            const bool drop = d == v0 || (mlo > 1 && d == v1) || (mlo > 2 && d == v2);
            __syncwarp();  // every lane has read its entry
            if (live && lane < 32 && !drop) F[lane + ins - can - shift] = d;
            // inserted entry k lands after the q_k entries below it, the
            // k - E_{<k} insertions before it, less the E_{<k} cancelled entries
            if (lane < mlo) {
                const int k = lane;
                const uint64_t v = k == 0 ? v0 : (k == 1 ? v1 : v2);
                const int q = k == 0 ? q0 : (k == 1 ? q1 : q2);
                const int ek = k == 0 ? e0 : (k == 1 ? e1 : e2);
                const int eb = (k > 0 ? e0 : 0) + (k > 1 ? e1 : 0);
                if (!ek) F[q + k - 2 * eb - shift] = v;
            }
            __syncwarp();
            W.fh -= shift;
            return true;
        }
    }
    const uint64_t *D = &sm.f[W.fb][W.fh];
    const uint64_t mine = lane == 0 ? x1 : (lane == 1 ? x2 : x3);
    int myq = 0, myeq = 0;
    if (lane < mlo) {
        int lo = 0, hi = nd;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (D[mid] < mine) lo = mid + 1; else hi = mid;
        }
        myq = lo;
        myeq = (lo < nd && D[lo] == mine) ? 1 : 0;
    }
    const int eq0 = __shfl_sync(0xFFFFFFFFu, myeq, 0), eq1 = __shfl_sync(0xFFFFFFFFu, myeq, 1),
              eq2 = __shfl_sync(0xFFFFFFFFu, myeq, 2);
    const int n2 = nd + mlo - 2 * (eq0 + (mlo > 1 ? eq1 : 0) + (mlo > 2 ? eq2 : 0));
    const int off = min(FRONT_SLACK, FCAP - n2);
    uint64_t *out = sm.f[W.fb ^ 1] + off;
    for (int i = lane; i < nd; i += 32) {
        const uint64_t d = D[i];
        int ins = 0, can = 0;
        if (v0 < d) { if (eq0) can++; else ins++; }
        if (v1 < d) { if (eq1) can++; else ins++; }
        if (v2 < d) { if (eq2) can++; else ins++; }
        const bool drop = (v0 == d) | (v1 == d) | (v2 == d);
        if (!drop) out[i + ins - can] = d;
    }
    if (lane < mlo && !myeq) {
        const int before_c = (lane > 0 ? eq0 : 0) + (lane > 1 ? eq1 : 0);
        out[myq + (lane - before_c) - before_c] = mine;
    }
    __syncwarp();
    W.fb ^= 1;
    W.fh = off;
    W.fn = off + n2;
    return true;
}

// Toggle the sorted, distinct entries X[0..n) (all above the removed pivot),
// read from shared memory or, XG, from the arena.  Entries up to tau are
// merged into the front (tau is lowered first if the front would overflow),
// a short rest goes to the inbox, a long rest straight into middle or base.
template <bool XG>
__device__ bool toggle_list(const RedParams &R, Work &W, WarpSmem &sm, const uint64_t *X, int n, RedStats &st) {
    const int lane = threadIdx.x & 31;
    // entries <= t: 32 evenly spaced probes per round narrow [lo, hi] 32-fold,
    // so a run in global memory costs a few round trips, not one per halving
    auto count_le = [&](uint64_t t) {
        int lo = 0, hi = n;
        while (hi - lo > 32) {
            const int step = (hi - lo + 31) / 32;
            const int idx = lo + lane * step;
            const unsigned m = __ballot_sync(0xFFFFFFFFu, idx < hi && (XG ? ld_cg(X + idx) : X[idx]) <= t);
            const int cnt = __popc(m);  // a prefix of the lanes
            if (cnt == 0) return lo;
            const int nhi = min(hi, lo + cnt * step);
            lo += (cnt - 1) * step + 1;
            hi = nhi;
        }
        const unsigned m = __ballot_sync(0xFFFFFFFFu, lo + lane < hi && (XG ? ld_cg(X + lo + lane) : X[lo + lane]) <= t);
        return lo + __popc(m);
    };
    int nlo = count_le(W.tau);
    if (nlo > 0 && W.fn - W.fh + nlo > FCAP) {
        uint64_t t = ~0ull;
        if (W.fn - W.fh > FCAP / 4) t = sm.f[W.fb][W.fh + FCAP / 4 - 1];
        if (nlo > FCAP / 4) {
            const uint64_t u = XG ? ld_cg(X + FCAP / 4 - 1) : X[FCAP / 4 - 1];
            t = u < t ? u : t;
        }
        if (!lower_tau(R, W, sm, t, st)) return false;
        nlo = count_le(W.tau);
    }
    if (nlo > 0) {
        const uint64_t *D = X;
        if (XG) {
#pragma unroll 8
            for (int k = lane; k < nlo; k += 32) sm.c[k] = ld_cg(X + k);
            __syncwarp();
            D = sm.c;
        }
        const int nf = insert_merge<false>(&sm.f[W.fb][W.fh], W.fn - W.fh, D, nlo, sm.f[W.fb ^ 1], sm);
        W.fb ^= 1;
        W.fh = 0;
        W.fn = nf;
    }
    const int nhi = n - nlo;
    if (nhi == 0) return true;
    const uint64_t *Xh = X + nlo;
    if (nhi <= ICAP) {
        if (W.ni + nhi > ICAP && !flush_inbox(R, W, sm, st)) return false;
        for (int k = lane; k < nhi; k += 32) sm.in[W.ni + k] = XG ? ld_cg(Xh + k) : Xh[k];
        W.ni += nhi;
        __syncwarp();
        return true;
    }
    // a long rest
    if (!flush_inbox(R, W, sm, st)) return false;
    if (W.mid_on && nhi <= MIDMAX) {
        const int nmid = W.nm - W.mstart, x = W.mown ^ 1;
        const int r = tiled_xor<true, XG>(W.mg[W.mown] + W.mstart, nmid, Xh, nhi, W.mg[x], MIDCAP, sm);
        __threadfence_block();
        if (r < 0) return false;
        W.mown = x;
        W.nm = r;
        W.mstart = 0;
        st.merged += (unsigned long long)(nmid + nhi);
        if (W.nm > MIDMAX && !merge_mid(R, W, sm, st)) return false;
        return true;
    }
    if (W.mid_on && !merge_mid(R, W, sm, st)) return false;
    const int na = W.nb - W.start;
    const uint64_t *A = W.g[W.bown] + W.start;
    if ((int64_t)na + nhi > W.cap && !grow_to(R, W, (int64_t)na + nhi)) return false;
    const int x = W.bown ^ 1;
    const int r = tiled_xor<true, XG>(A, na, Xh, nhi, W.g[x], W.cap, sm);
    __threadfence_block();
    if (r < 0) return false;
    W.bown = x;
    W.nb = r;
    W.start = 0;
    st.merged += (unsigned long long)(na + nhi);
    return true;
}

// Place of cofacet g (0..3) of the edge along axis a at c, in the order the
// cofacets are formed above (+b1, -b1, +b2, -b2 faces): its type t, its anchor
// ac and its L; false if it lies outside the image.  No values are needed.
__device__ __forceinline__ bool edge_cofacet_place(const Seg &S, int a, const int *c, int g, int &t, int *ac,
                                                   uint32_t &L) {
    const int b = g < 2 ? (a == 0 ? 1 : 0) : (a == 2 ? 1 : 2);
    const bool minus = (g & 1) != 0;
    const int cb = b == 0 ? c[0] : (b == 1 ? c[1] : c[2]);
    const int nb = b == 0 ? S.nx : (b == 1 ? S.ny : S.nz);
    ac[0] = c[0] - (minus && b == 0);
    ac[1] = c[1] - (minus && b == 1);
    ac[2] = c[2] - (minus && b == 2);
    t = min(a, b) + max(a, b) - 1;
    L = cube_L(S, t, ac[0], ac[1], ac[2]);
    return minus ? cb >= 1 : cb + 1 < nb;
}

// The lookahead entry of face `cand` (type fm, anchor c) from the results of
// its first round trip: the code bytes k0, k1 of the two edges that could pair
// it as apparent and its pivot-table word pe.  L.key, L.kind = 0 and L.k = 0
// are set by the caller.
__device__ void look_finish(const RedParams &R, const Seg &S, uint64_t cand, int fm, const int *c, uint32_t k0,
                            uint32_t k1, unsigned long long pe, Look &L) {
    int ea = -1, ec[3] = {c[0], c[1], c[2]};
    if (fm == 2) {
        if (((k0 >> 3) & 3u) == 1u) ea = 1;
        else if (((k1 >> 3) & 3u) == 2u) { ea = 1; ec[2] += 1; }
    } else if (fm == 1) {
        if ((k0 & 7u) == 1u) ea = 0;
        else if ((k1 & 7u) == 2u) { ea = 0; ec[2] += 1; }
    } else {
        if ((k0 & 7u) == 3u) ea = 0;
        else if ((k1 & 7u) == 4u) { ea = 0; ec[1] += 1; }
    }
    // the second round trip: the apparent edge's vertex values, or the
    // owner's version (its header and first four entries; the arena keeps
    // ARENA_SLACK words of slack past its last version), issued together
    const bool owned = ea < 0 && pe != PIV_FREE;
    uint64_t vn = 0, vh = 0, a1 = 0, a2 = 0, a3 = 0;
    if (owned) {
        const uint64_t *C = R.arena + piv_off(pe);
        vn = ld_cg(C);
        vh = ld_cg(C + 1);
        a1 = ld_cg(C + 2);
        a2 = ld_cg(C + 3);
        a3 = ld_cg(C + 4);
    }
    if (ea >= 0) {
        // the apparent edge's column: its cofacets, the face itself first
        uint64_t f0, f1, f2, f3;
        L.k = edge_cofacets_sorted(R.I, S, ea, ec, f0, f1, f2, f3);
        L.kind = 1;
        L.c1 = f1;
        L.c2 = f2;
        L.c3 = f3;
        return;
    }
    if (!owned) return;
    L.kind = 2;
    L.own = piv_owner(pe);
    L.ver = pe;
    if (vn >= 1 && vn <= 4 && vh == cand) {
        L.c1 = vn > 1 ? a1 : ~0ull;
        L.c2 = vn > 2 ? a2 : ~0ull;
        L.c3 = vn > 3 ? a3 : ~0ull;
        L.k = (int)vn;
    }
}


// Fill the lookahead cache for the front's next 32 entries in two round
// trips: the code bytes of the two edges that could pair the face as
// apparent and its pivot-table entry, then either the apparent edge's vertex
// values (its column is generated from them) or the head of the owner's
// version.
__device__ void look_refill(const RedParams &R, const Seg &S, const Work &W, const WarpSmem &sm, Look &L) {
    const int lane = threadIdx.x & 31;
    const uint64_t cand = W.fh + lane < W.fn ? sm.f[W.fb][W.fh + lane] : ~0ull;
    L.key = cand;
    L.kind = 0;
    L.k = 0;
    if (cand == ~0ull) return;
    const uint32_t fl = key_L(cand);
    const int64_t bit = S.loff + fl;
    // the face's type and anchor voxel need no division (L = type * P + voxel),
    // so the first loads go out before the anchor's coordinates are decoded
    const uint32_t P3 = (uint32_t)S.nx * (uint32_t)S.ny * (uint32_t)S.nz;
    const int fm = (fl >= P3) + (fl >= 2u * P3);
    // the two edges that could pair this face as apparent (the code bytes of
    // their voxels): {x,z} (type 1) the x-edges at c (+z) and c+z (-z); {x,y}
    // (type 0) the x-edges at c (+y) and c+y (-y); {y,z} (type 2) the y-edges
    // at c (+z) and c+z (-z)
    const int64_t v0 = S.voff + (int64_t)(fl - (uint32_t)fm * P3);
    const int64_t v1 = v0 + (fm == 0 ? (int64_t)S.nx : (int64_t)S.nx * S.ny);
    const uint32_t k0 = R.I.code[v0], k1 = R.I.code[v1];
    const unsigned long long pe = __ldcg(&R.P[bit]);
    int fm2, c[3];
    decode_L(S, fl, fm2, c);  // fm2 == fm
    look_finish(R, S, cand, fm, c, k0, k1, pe, L);
}

// publish the working column as column j's current version; *voff is the
// arena offset of its header (for the pivot-table entry)
__device__ bool publish_work(const RedParams &R, int64_t j, Work &W, WarpSmem &sm, RedStats &st,
                             unsigned long long *voff) {
    const int lane = threadIdx.x & 31;
    const bool levels = W.nb - W.start > 0 || (W.mid_on && W.nm - W.mstart > 0);
    const uint64_t *rest;
    int nrest;
    if (!levels) {
        W.ni = sort_inbox(sm, W.ni);  // still the inbox (its order is free)
        rest = sm.in;
        nrest = W.ni;
    } else {
        if (!flush_inbox(R, W, sm, st)) return false;
        if (W.mid_on && W.nm - W.mstart > 0 && !merge_mid(R, W, sm, st)) return false;
        rest = W.g[W.bown] + W.start;
        nrest = W.nb - W.start;
    }
    const int nf = W.fn - W.fh, n = nf + nrest;
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(R.arena_top, (unsigned long long)(n + 1));
    off = __shfl_sync(0xFFFFFFFFu, off, 0);
    if ((int64_t)(off + n + 1) > R.arena_cap || off > PIV_OFF_MASK) return false;
    if (lane == 0) __stcg((unsigned long long *)&R.arena[off], (unsigned long long)n);
    for (int k = lane; k < nf; k += 32) __stcg((unsigned long long *)&R.arena[off + 1 + k], sm.f[W.fb][W.fh + k]);
    for (int k = lane; k < nrest; k += 32)
        __stcg((unsigned long long *)&R.arena[off + 1 + nf + k], levels ? ld_cg(rest + k) : rest[k]);
    // the entries are visible before the pivot-table entry that names them
    // (the caller's CAS); the column's current version is read only after
    // the kernel, by the emission of the pairs
    __threadfence();
    __syncwarp();
    if (lane == 0) R.cur[j] = (off << 24) | (unsigned long long)n;
    __syncwarp();
    *voff = off;
    return true;
}

// One warp per column.  With R.resume the columns are those an earlier pass
// set aside (their published versions); with R.budget > 0 a column still
// unsettled after that many iterations is published and set aside.
__global__ void __launch_bounds__(RED_WARPS * 32, RED_BLOCKS) k_h1_reduce(RedParams R) {
    extern __shared__ __align__(16) unsigned char red_smem[];
    WarpSmem *smem = reinterpret_cast<WarpSmem *>(red_smem);
    const int lane = threadIdx.x & 31;
    WarpSmem &sm = smem[threadIdx.x >> 5];
    RedStats st;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    Work W;
    Look look;
    W.g[0] = R.scratch + wid * 2 * (int64_t)R.maxlen;
    W.g[1] = W.g[0] + R.maxlen;
    W.cap = R.maxlen;
    W.mg[0] = W.mg[1] = nullptr;
    W.mid_on = false;
    const int64_t CAP = R.cap;
    TSTAMP_KERNEL(R);
    const int64_t items = R.resume ? (int64_t)min(*R.dcount, (unsigned long long)R.dcap) : R.ncols;
    for (;;) {
        unsigned long long jj = 0;
        if (lane == 0) jj = atomicAdd(R.resume ? R.dnext : R.next, 1ull);
        jj = __shfl_sync(0xFFFFFFFFu, jj, 0);
        if ((int64_t)jj >= items) { flush_stats(R, st); return; }
        TSTAMP_COLSTART(col_t0);
        int64_t j = (int64_t)jj;
        unsigned long long dver = 0;
        if (R.resume) {
            const unsigned long long e = R.dlist[jj];
            j = piv_owner(e);
            dver = piv_off(e);
        }
        const uint64_t jkey = R.colkey[j];
        const Seg S = R.segs[R.colseg[j]];
        W.fb = 0;
        W.fh = 0;
        W.tau = ~0ull;
        W.ni = 0;
        W.bown = 0;
        W.nb = W.start = 0;
        W.mid_on = false;
        W.nm = W.mstart = 0;
        if (!R.resume) {
            // the coboundary of edge j is the front; nothing lies beyond it
            int a, c[3];
            decode_L(S, key_L(jkey), a, c);
            // lanes 0..3 read the code bytes and pivot-table word of one cofacet
            // each, in the round trip that reads the vertex values: a cofacet's
            // place needs no values
            int gt = 0, gc[3] = {0, 0, 0};
            uint32_t gL = 0, gk0 = 0, gk1 = 0;
            unsigned long long gpe = PIV_FREE;
            int gok = 0;
            if (lane < 4) {
                gok = edge_cofacet_place(S, a, c, lane, gt, gc, gL) ? 1 : 0;
                if (gok) {
                    const int64_t v0 = S.voff + ((int64_t)gc[2] * S.ny + gc[1]) * S.nx + gc[0];
                    const int64_t v1 = v0 + (gt == 0 ? (int64_t)S.nx : (int64_t)S.nx * S.ny);
                    gk0 = R.I.code[v0];
                    gk1 = R.I.code[v1];
                    gpe = __ldcg(&R.P[S.loff + gL]);
                }
            }
            uint64_t f0, f1, f2, f3;
            const int k = edge_cofacets_sorted(R.I, S, a, c, f0, f1, f2, f3);
            const uint64_t fr = lane == 0 ? f0 : (lane == 1 ? f1 : (lane == 2 ? f2 : f3));
            if (lane < k) sm.f[0][lane] = fr;
            W.fn = k;
            // the lookahead of the front: lane r < k takes what was read for the
            // cofacet that sorts r-th (faces have distinct L)
            const uint32_t Lr = key_L(fr);
            int src = 0;
#pragma unroll
            for (int g = 0; g < 4; g++) {
                const uint32_t Lg = __shfl_sync(0xFFFFFFFFu, gL, g);
                const int okg = __shfl_sync(0xFFFFFFFFu, gok, g);
                if (okg && Lg == Lr) src = g;
            }
            const int rt = __shfl_sync(0xFFFFFFFFu, gt, src);
            const int rc[3] = {__shfl_sync(0xFFFFFFFFu, gc[0], src), __shfl_sync(0xFFFFFFFFu, gc[1], src),
                               __shfl_sync(0xFFFFFFFFu, gc[2], src)};
            const uint32_t rk0 = __shfl_sync(0xFFFFFFFFu, gk0, src), rk1 = __shfl_sync(0xFFFFFFFFu, gk1, src);
            const unsigned long long rpe = __shfl_sync(0xFFFFFFFFu, gpe, src);
            look.key = lane < k ? fr : ~0ull;
            look.kind = 0;
            look.k = 0;
            if (lane < k) look_finish(R, S, fr, rt, rc, rk0, rk1, rpe, look);
            __syncwarp();
        } else {
            // the version the earlier pass published becomes the working column
            W.fn = 0;
            const int len = (int)ld_cg(R.arena + dver);
            if (!toggle_list<true>(R, W, sm, R.arena + dver + 1, len, st)) {
                if (lane == 0) fail_ws(R.status, SITE_POOL);
                flush_stats(R, st);
                return;
            }
            look.key = ~0ull;
            look.kind = 0;
        }
        int64_t it = 0;
        bool keep = R.budget <= 0;  // no budget, or no room left to set the column aside
        for (;;) {
            if (++it > CAP) { if (lane == 0) set_status(R.status, CR_ERR_TIMEOUT); flush_stats(R, st); return; }
            st.it++;
            if ((unsigned long long)it > st.maxit) st.maxit = (unsigned long long)it;
            st.lng = it > 16384;
            TITER(st);
#ifdef CR_H1_TIMING
            if (st.lng) st.t[7]++;
#endif
            if (!front_ready(R, W, sm, st)) {
                if (lane == 0) fail_ws(R.status, SITE_POOL);
                flush_stats(R, st);
                return;
            }
            if (W.fh == W.fn) { if (lane == 0) set_status(R.status, CR_ERR_INTERNAL); break; }
            // over budget, or the queue is drained (then the rest of the pass
            // would run at this instance's lower speed per column): publish the
            // column as it stands and set it aside
            if (!keep && (it > R.budget || ((it & 31) == 0 && __shfl_sync(0xFFFFFFFFu, __ldcg(R.next), 0) >= (unsigned long long)R.ncols))) {
                unsigned long long voff = 0;
                if (!publish_work(R, j, W, sm, st, &voff)) { if (lane == 0) fail_ws(R.status, SITE_ARENA); flush_stats(R, st); return; }
                unsigned long long di = 0;
                if (lane == 0) di = atomicAdd(R.dcount, 1ull);
                di = __shfl_sync(0xFFFFFFFFu, di, 0);
                if ((int64_t)di < R.dcap) {
                    if (lane == 0) R.dlist[di] = piv_make(j, voff);
                    break;
                }
                keep = true;
            }
            const uint64_t p = sm.f[W.fb][W.fh];
            const int64_t gidx = S.loff + key_L(p);
            TMARK(t1);
            unsigned hit = __ballot_sync(0xFFFFFFFFu, look.key == p);
            if (!hit) {
#ifdef CR_H1_TIMING
                if (st.lng) st.t[6]++;
#endif
                look_refill(R, S, W, sm, look);  // p is lane 0's entry
                hit = __ballot_sync(0xFFFFFFFFu, look.key == p);
            }
            const int hl = hit ? __ffs(hit) - 1 : 0;
            const int hkind = hit ? __shfl_sync(0xFFFFFFFFu, look.kind, hl) : 0;
            const uint64_t c1 = __shfl_sync(0xFFFFFFFFu, look.c1, hl), c2 = __shfl_sync(0xFFFFFFFFu, look.c2, hl),
                           c3 = __shfl_sync(0xFFFFFFFFu, look.c3, hl);
            const int hk = __shfl_sync(0xFFFFFFFFu, look.k, hl), hown = __shfl_sync(0xFFFFFFFFu, look.own, hl);
            const unsigned long long hver = __shfl_sync(0xFFFFFFFFu, look.ver, hl);
            if (hit && lane == hl) look.key = ~0ull;  // used once
            TADD(st, 1, t1);
            if (hkind == 1) {
                st.app++;
                TMARK(t2);
                W.fh++;
                const bool okadd = toggle_small(R, W, sm, c1, c2, c3, hk - 1, st);
                TADD(st, 2, t2);
                if (!okadd) {
                    if (lane == 0) fail_ws(R.status, SITE_POOL);
                    flush_stats(R, st);
                    return;
                }
                continue;
            }
            TMARK(t9);
            // a pivot the lookahead found free is claimed without reading the
            // table again: if it has been taken since, the claim fails and the
            // step is retried with a fresh lookup
            const unsigned long long pe = hkind == 2 ? hver : (hit && hkind == 0 ? PIV_FREE : __ldcg(&R.P[gidx]));
            const int o = hkind == 2 ? hown : piv_owner(pe);
#ifdef CR_H1_TIMING
            if (hkind != 2) (void)__shfl_sync(0xFFFFFFFFu, (int)pe, 0);  // make the read complete here
#endif
            TADD(st, 9, t9);
            if (o < 0) {
                unsigned long long voff = 0;
                if (!publish_work(R, j, W, sm, st, &voff)) { if (lane == 0) fail_ws(R.status, SITE_ARENA); flush_stats(R, st); return; }
                unsigned long long prev = 0;
                if (lane == 0) prev = atomicCAS(&R.P[gidx], PIV_FREE, piv_make(j, voff));
                prev = __shfl_sync(0xFFFFFFFFu, prev, 0);
                if (prev == PIV_FREE) break;  // j settled
                st.retry++;
                continue;
            }
            if ((int64_t)o == j) break;
            // columns are numbered in cohomology order: a smaller index is an earlier column
            const bool takeover = (int64_t)o > j;  // o is a later column: j takes its pivot, then continues with o
            if (takeover) {
                unsigned long long voff = 0;
                if (!publish_work(R, j, W, sm, st, &voff)) { if (lane == 0) fail_ws(R.status, SITE_ARENA); flush_stats(R, st); return; }
                unsigned long long prev = 0;
                if (lane == 0) prev = atomicCAS(&R.P[gidx], pe, piv_make(j, voff));
                prev = __shfl_sync(0xFFFFFFFFu, prev, 0);
                if (prev != pe) { st.retry++; continue; }
                st.take++;
                look.key = ~0ull;  // snapshots taken for column j's pivots
            }
            TMARK(t3);
            if (hkind == 2 && !takeover && hk > 0) {
                // the snapshot's version is short and was read with the fill
                st.add++;
                W.fh++;
                const bool okadd = toggle_small(R, W, sm, c1, c2, c3, hk - 1, st);
                TADD(st, 3, t3);
                if (!okadd) {
                    if (lane == 0) fail_ws(R.status, SITE_POOL);
                    flush_stats(R, st);
                    return;
                }
                continue;
            }
            // the version of o with pivot p that the pivot-table entry names:
            // its header and first 31 entries in one round trip
            const uint64_t *V = R.arena + piv_off(pe);
            const uint64_t w = ld_cg(V + lane);
            const int len = (int)__shfl_sync(0xFFFFFFFFu, w, 0);
            if (len == 0) continue;
            bool ok2;
            if (len - 1 <= DMAX) {
                if (lane >= 1 && lane <= len) sm.c[lane - 1] = w;
#pragma unroll 8
                for (int q2 = 31 + lane; q2 < len; q2 += 32) sm.c[q2] = ld_cg(V + 1 + q2);
                __syncwarp();
                if (sm.c[0] != p) { st.retry++; continue; }
                st.add++;
                TMARK(t4);
                W.fh++;
                ok2 = toggle_list<false>(R, W, sm, sm.c + 1, len - 1, st);
                TADD(st, 4, t4);
            } else {
                if (__shfl_sync(0xFFFFFFFFu, w, 1) != p) { st.retry++; continue; }
                st.add++;
                TMARK(t4);
                W.fh++;
                ok2 = toggle_list<true>(R, W, sm, V + 2, len - 1, st);
                TADD(st, 4, t4);
            }
            if (!ok2) {
                if (lane == 0) fail_ws(R.status, SITE_POOL);
                flush_stats(R, st);
                return;
            }
            if (takeover) j = o;
        }
        TSTAMP_COLEND(R, it, col_t0);
    }
}

