// pmp_exchange.cu -- the batched form on several ranks (host side): patches
// assigned to ranks along a space-filling curve, and the plan of what each
// rank holds and exchanges with its neighbours in a pass (Sec. 2.2, Step 2:
// the ghost zones of a buffer that lie on another rank's cells are sent to
// that rank and added there in the fixed order of App. A.2).
//
// A rank keeps its owned patches, one proxy per patch of another rank that
// neighbours one of them, and a zero patch.  The proxies make the owned
// patches' work exactly that of the one-rank batched pass: their valid state
// cells carry the neighbour's state where the owned patches' ghost zones read
// it, their buffer ghost cells the neighbour's deposits that fall on owned
// cells (the images the App. A.2 sum adds, in the same order), and for sinks
// their valid buffer cells the neighbour's folded sums where Step 4 of an
// owned sink reads eta.  Everything here is host code: it runs without a GPU.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "pmp.h"

namespace {

constexpr int kNF = 5;

// Offsets (ox, oy, oz) of the 26 neighbours, oz slowest, ox fastest.
void offset_of(int t, int o[3])
{
    const int u = t < 13 ? t : t + 1;
    o[0] = u % 3 - 1;
    o[1] = (u / 3) % 3 - 1;
    o[2] = u / 9 - 1;
}

int slot_of(int ox, int oy, int oz)
{
    const int t = ((oz + 1) * 3 + (oy + 1)) * 3 + (ox + 1);
    return t > 13 ? t - 1 : t;
}

unsigned long long spread3(unsigned v)
{
    unsigned long long x = v & 0x1fffffULL;
    x = (x | (x << 32)) & 0x1f00000000ffffULL;
    x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}

struct Box {
    int patch;  // global index
    int lo[3], hi[3];
    bool operator==(const Box &b) const
    {
        return patch == b.patch && std::memcmp(lo, b.lo, sizeof(lo)) == 0 && std::memcmp(hi, b.hi, sizeof(hi)) == 0;
    }
};

long long volume(const int lo[3], const int hi[3])
{
    return (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
}

}  // namespace

struct pmp_plan {
    int rank, n_ranks, ng, n_owned, n_local;
    std::vector<pmp_patch> local;
    std::vector<int32_t> gid;
    long long arena_len;
    // [kind][send] region lists, offsets absolute in one buffer holding the
    // peer messages one after the other in increasing peer rank
    std::vector<pmp_region> regions[3][2];
};

namespace {

// Boxes of patches owned by `sender` that the receiver needs, in the order
// both sides enumerate (receiver's patches in global order, then the 26
// offsets), each distinct box once.
//   STATE, FOLDED: for each patch p of the receiver and neighbour q = nb[p][o]
//     of the sender, q's valid cells in p's ghost zone.
//   GHOST: for each patch q of the receiver and image offset o, the patch
//     p = nb[q][-o] of the sender holds q's images in its ghost cells.
std::vector<Box> needed(const pmp_patch *P, int np, int ng, const int32_t *rank_of, int receiver, int sender, int kind)
{
    std::vector<Box> out;
    for (int p = 0; p < np; ++p) {
        if (rank_of[p] != receiver) continue;
        for (int t = 0; t < 26; ++t) {
            int o[3];
            offset_of(t, o);
            Box b;
            if (kind == PMP_XCH_GHOST) {
                const int q = P[p].neighbour[slot_of(-o[0], -o[1], -o[2])];
                if (rank_of[q] != sender) continue;
                b.patch = q;
                for (int a = 0; a < 3; ++a) {
                    const int n = P[q].n[a];
                    b.lo[a] = o[a] > 0 ? n : (o[a] < 0 ? -ng : 0);
                    b.hi[a] = o[a] > 0 ? n + ng : (o[a] < 0 ? 0 : n);
                }
            } else {
                const int q = P[p].neighbour[t];
                if (rank_of[q] != sender) continue;
                b.patch = q;
                for (int a = 0; a < 3; ++a) {
                    const int n = P[q].n[a];
                    b.lo[a] = o[a] < 0 ? n - ng : 0;
                    b.hi[a] = o[a] > 0 ? ng : n;
                }
            }
            if (std::find(out.begin(), out.end(), b) == out.end()) out.push_back(b);
        }
    }
    return out;
}

}  // namespace

extern "C" {

pmp_status pmp_partition_sfc(int32_t n_patches, const int32_t *pos, const int64_t *cost, int32_t n_ranks,
                             int32_t *rank_of)
{
    if (n_patches < 1 || !pos || !cost || n_ranks < 1 || !rank_of) return PMP_ERR_ARG;
    long double total = 0.0L;
    for (int p = 0; p < n_patches; ++p) {
        for (int a = 0; a < 3; ++a)
            if (pos[3 * p + a] < 0 || pos[3 * p + a] >= (1 << 20)) return PMP_ERR_ARG;
        if (cost[p] < 1) return PMP_ERR_ARG;
        total += (long double)cost[p];
    }
    std::vector<int> order(n_patches);
    for (int p = 0; p < n_patches; ++p) order[p] = p;
    auto key = [&](int p) {
        return spread3((unsigned)pos[3 * p]) | (spread3((unsigned)pos[3 * p + 1]) << 1) |
               (spread3((unsigned)pos[3 * p + 2]) << 2);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return key(x) < key(y); });
    // cut the curve where the cumulative cost passes r / n_ranks of the total
    // (at the nearer patch boundary); every rank gets at least one patch when
    // there are enough patches
    long double acc = 0.0L;
    int r = 0;
    for (int i = 0; i < n_patches; ++i) {
        const int p = order[i];
        const long double mid = acc + 0.5L * (long double)cost[p];
        int want = (int)(mid * n_ranks / total);
        if (want > n_ranks - 1) want = n_ranks - 1;
        if (want < r) want = r;
        // no rank skipped: a patch that carries more than 1 / n_ranks of the
        // cost would otherwise carry the cut past the next rank
        const int next = i == 0 ? 0 : r + 1;
        if (want > next) want = next;
        // leave at least one patch for each later rank
        const int left = n_patches - i;
        if (n_ranks - want > left) want = n_ranks - left;
        r = want;
        rank_of[p] = r;
        acc += (long double)cost[p];
    }
    return PMP_OK;
}

pmp_status pmp_plan_create(const pmp_patch *patches, int32_t n_patches, int32_t ng, const int32_t *rank_of,
                           int32_t n_ranks, int32_t rank, pmp_plan **out)
{
    if (!out) return PMP_ERR_ARG;
    *out = nullptr;
    if (!patches || n_patches < 1 || ng < 0 || !rank_of || n_ranks < 1 || rank < 0 || rank >= n_ranks)
        return PMP_ERR_ARG;
    for (int p = 0; p < n_patches; ++p) {
        if (rank_of[p] < 0 || rank_of[p] >= n_ranks) return PMP_ERR_ARG;
        for (int a = 0; a < 3; ++a)
            if (patches[p].n[a] < ng || patches[p].n[a] < 1 || patches[p].n[a] + 2LL * ng > 0x1fffff) return PMP_ERR_ARG;
        for (int t = 0; t < 26; ++t)
            if (patches[p].neighbour[t] < 0 || patches[p].neighbour[t] >= n_patches) return PMP_ERR_ARG;
    }
    pmp_plan *pl = new (std::nothrow) pmp_plan();
    if (!pl) return PMP_ERR_ARG;
    pl->rank = rank;
    pl->n_ranks = n_ranks;
    pl->ng = ng;
    // local patches: owned, proxies, the zero patch
    std::vector<int> local_of(n_patches, -1);
    for (int p = 0; p < n_patches; ++p)
        if (rank_of[p] == rank) {
            local_of[p] = (int)pl->gid.size();
            pl->gid.push_back(p);
        }
    pl->n_owned = (int)pl->gid.size();
    std::vector<char> is_proxy(n_patches, 0);
    for (int i = 0; i < pl->n_owned; ++i)
        for (int t = 0; t < 26; ++t) {
            const int q = patches[pl->gid[i]].neighbour[t];
            if (rank_of[q] != rank) is_proxy[q] = 1;
        }
    for (int q = 0; q < n_patches; ++q)
        if (is_proxy[q]) {
            local_of[q] = (int)pl->gid.size();
            pl->gid.push_back(q);
        }
    const int zero = (int)pl->gid.size();
    pl->gid.push_back(-1);
    pl->n_local = zero + 1;
    int zn[3] = {ng > 0 ? ng : 1, ng > 0 ? ng : 1, ng > 0 ? ng : 1};
    for (int p = 0; p < n_patches; ++p)
        for (int a = 0; a < 3; ++a) zn[a] = std::max(zn[a], (int)patches[p].n[a]);
    long long off = 0;
    pl->local.resize(pl->n_local);
    for (int i = 0; i < pl->n_local; ++i) {
        pmp_patch &lp = pl->local[i];
        std::memset(&lp, 0, sizeof(lp));
        const int gp = pl->gid[i];
        for (int a = 0; a < 3; ++a) lp.n[a] = gp >= 0 ? patches[gp].n[a] : zn[a];
        for (int t = 0; t < 26; ++t) lp.neighbour[t] = (i < pl->n_owned) ? local_of[patches[gp].neighbour[t]] : zero;
        const long long pc = ((long long)lp.n[0] + 2 * ng) * ((long long)lp.n[1] + 2 * ng) * ((long long)lp.n[2] + 2 * ng);
        lp.field_stride = (pc + 31) / 32 * 32;
        lp.offset = off;
        off += kNF * lp.field_stride;
    }
    pl->arena_len = off;
    // region lists: peer after peer, send lists enumerated as the peer
    // enumerates its receive lists
    for (int kind = 0; kind < 3; ++kind) {
        long long base[2] = {0, 0};
        for (int peer = 0; peer < n_ranks; ++peer) {
            if (peer == rank) continue;
            for (int send = 0; send < 2; ++send) {
                const std::vector<Box> bx = send ? needed(patches, n_patches, ng, rank_of, peer, rank, kind)
                                                 : needed(patches, n_patches, ng, rank_of, rank, peer, kind);
                for (const Box &b : bx) {
                    pmp_region r;
                    std::memset(&r, 0, sizeof(r));
                    r.peer = peer;
                    r.patch = local_of[b.patch];
                    for (int a = 0; a < 3; ++a) {
                        r.lo[a] = b.lo[a];
                        r.hi[a] = b.hi[a];
                    }
                    r.offset = base[send];
                    base[send] += kNF * volume(b.lo, b.hi);
                    pl->regions[kind][send].push_back(r);
                }
            }
        }
    }
    *out = pl;
    return PMP_OK;
}

pmp_status pmp_plan_local(const pmp_plan *plan, int32_t *n_owned, int32_t *n_local, pmp_patch *local,
                          int32_t *global_id, int64_t *arena_len)
{
    if (!plan) return PMP_ERR_ARG;
    if (n_owned) *n_owned = plan->n_owned;
    if (n_local) *n_local = plan->n_local;
    if (arena_len) *arena_len = plan->arena_len;
    for (int i = 0; i < plan->n_local; ++i) {
        if (local) local[i] = plan->local[i];
        if (global_id) global_id[i] = plan->gid[i];
    }
    return PMP_OK;
}

pmp_status pmp_plan_regions(const pmp_plan *plan, int32_t kind, int32_t send, pmp_region *out, int32_t max,
                            int32_t *n)
{
    if (!plan || kind < 0 || kind > 2 || (send != 0 && send != 1) || !n || (max > 0 && !out)) return PMP_ERR_ARG;
    const std::vector<pmp_region> &v = plan->regions[kind][send];
    *n = (int32_t)v.size();
    for (int i = 0; i < (int)v.size() && i < max; ++i) out[i] = v[i];
    return PMP_OK;
}

void pmp_plan_destroy(pmp_plan *plan) { delete plan; }

}  // extern "C"
