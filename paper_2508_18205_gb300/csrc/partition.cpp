// partition.cpp -- node partitions and halo plans for a sharded step (host only).
//
// A shard owns a contiguous range of a node set taken in a given order (the
// Morton order keeps ranges compact in space, so halos stay thin). Every
// stencil sum at an owned centre (Eq. 16) reads owned nodes and halo nodes;
// the plan lists, for every pair of shards, which nodes travel in one
// exchange, and rewrites each stencil set into local indices over the array
// [owned values | halo values]. No CUDA call is made here.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

struct mfd_partition {
    int64_t n = 0;
    int nshards = 0;
    std::vector<int64_t> order;   // position -> caller id
    std::vector<int64_t> pos;     // caller id -> position
    std::vector<int32_t> owner;   // caller id -> shard
    std::vector<int64_t> start;   // nshards + 1 range starts (positions)
};

struct mfd_halo {
    int nshards = 0;
    int nsets = 0;
    std::vector<int64_t> src_start;           // range starts of the source partition
    // halo of shard s: caller ids, grouped by owner, partition order within a group
    std::vector<std::vector<int64_t>> halo;
    std::vector<std::vector<int64_t>> group;  // [s][nshards + 1] offsets of the owner groups
    // localised stencils: [set][shard] -> int32 rows of the owned centres
    std::vector<std::vector<std::vector<int32_t>>> local;
    std::vector<int> ncols;
};

namespace {

mfd_status check_part(const mfd_partition* p, const char* what) {
    if (!p) return mfd::fail(MFD_ERR_ARG, std::string(what) + ": null partition");
    return MFD_OK;
}

}  // namespace

extern "C" {

mfd_status mfd_partition_create(int64_t n, const int64_t* order, int nshards, mfd_partition** out) {
    if (!out) return mfd::fail(MFD_ERR_ARG, "mfd_partition_create: out is null");
    *out = nullptr;
    if (n < 0 || nshards < 1 || nshards > 65536)
        return mfd::fail(MFD_ERR_ARG, "mfd_partition_create: need n >= 0 and 1 <= nshards <= 65536");
    try {
        auto* p = new mfd_partition;
        p->n = n;
        p->nshards = nshards;
        p->order.resize(n);
        p->pos.assign(n, -1);
        for (int64_t r = 0; r < n; ++r) {
            int64_t id = order ? order[r] : r;
            if (id < 0 || id >= n || p->pos[id] >= 0) {
                delete p;
                return mfd::fail(MFD_ERR_ARG, "mfd_partition_create: order is not a permutation of 0..n-1");
            }
            p->order[r] = id;
            p->pos[id] = r;
        }
        p->start.resize(nshards + 1);
        for (int s = 0; s <= nshards; ++s) p->start[s] = (int64_t)((__int128)n * s / nshards);
        p->owner.resize(n);
        for (int s = 0; s < nshards; ++s)
            for (int64_t r = p->start[s]; r < p->start[s + 1]; ++r) p->owner[p->order[r]] = s;
        *out = p;
        return MFD_OK;
    } catch (const std::bad_alloc&) {
        return mfd::fail(MFD_ERR_OOM, "mfd_partition_create: host allocation failed");
    }
}

mfd_status mfd_partition_owner(const mfd_partition* part, int32_t* owner) {
    MFD_TRY(check_part(part, "mfd_partition_owner"));
    if (!owner && part->n) return mfd::fail(MFD_ERR_ARG, "mfd_partition_owner: owner is null");
    if (part->n) std::memcpy(owner, part->owner.data(), sizeof(int32_t) * part->n);
    return MFD_OK;
}

mfd_status mfd_partition_owned(const mfd_partition* part, int shard, int64_t* count, int64_t* ids) {
    MFD_TRY(check_part(part, "mfd_partition_owned"));
    if (!count || shard < 0 || shard >= part->nshards)
        return mfd::fail(MFD_ERR_ARG, "mfd_partition_owned: bad shard or null count");
    int64_t a = part->start[shard], b = part->start[shard + 1];
    *count = b - a;
    if (ids)
        for (int64_t r = a; r < b; ++r) ids[r - a] = part->order[r];
    return MFD_OK;
}

void mfd_partition_destroy(mfd_partition* part) { delete part; }

mfd_status mfd_halo_create(const mfd_partition* src, int nsets, const mfd_partition* const* centres,
                           const int* ncols, const int64_t* const* idx, mfd_halo** out) {
    if (!out) return mfd::fail(MFD_ERR_ARG, "mfd_halo_create: out is null");
    *out = nullptr;
    MFD_TRY(check_part(src, "mfd_halo_create"));
    if (nsets < 1 || nsets > 16 || !centres || !ncols || !idx)
        return mfd::fail(MFD_ERR_ARG, "mfd_halo_create: need 1 <= nsets <= 16 and non-null arrays");
    const int S = src->nshards;
    for (int k = 0; k < nsets; ++k) {
        MFD_TRY(check_part(centres[k], "mfd_halo_create"));
        if (centres[k]->nshards != S)
            return mfd::fail(MFD_ERR_ARG, "mfd_halo_create: centre and source partitions differ in shard count");
        if (ncols[k] < 1 || (!idx[k] && centres[k]->n))
            return mfd::fail(MFD_ERR_ARG, "mfd_halo_create: bad ncols or null idx");
        const int64_t tot = centres[k]->n * (int64_t)ncols[k];
        for (int64_t e = 0; e < tot; ++e)
            if (idx[k][e] < 0 || idx[k][e] >= src->n)
                return mfd::fail(MFD_ERR_ARG, "mfd_halo_create: stencil entry outside the source set");
    }
    try {
        auto* h = new mfd_halo;
        h->nshards = S;
        h->nsets = nsets;
        h->src_start = src->start;
        h->ncols.assign(ncols, ncols + nsets);
        h->halo.resize(S);
        h->group.resize(S);
        h->local.assign(nsets, std::vector<std::vector<int32_t>>(S));
        // slot[pos] = local index of the source node at that position for the
        // shard being built (stamped per shard), so each shard costs O(its
        // stencil entries + its halo log halo)
        std::vector<int64_t> slot(src->n, -1);
        std::vector<int32_t> stamp(src->n, -1);
        for (int s = 0; s < S; ++s) {
            const int64_t own_a = src->start[s], own_b = src->start[s + 1];
            const int64_t n_own = own_b - own_a;
            std::vector<int64_t> hpos;  // halo positions (partition order), unsorted
            for (int k = 0; k < nsets; ++k) {
                const mfd_partition* c = centres[k];
                for (int64_t r = c->start[s]; r < c->start[s + 1]; ++r) {
                    const int64_t* row = idx[k] + c->order[r] * (int64_t)ncols[k];
                    for (int j = 0; j < ncols[k]; ++j) {
                        int64_t p = src->pos[row[j]];
                        if ((p < own_a || p >= own_b) && stamp[p] != s) {
                            stamp[p] = s;
                            hpos.push_back(p);
                        }
                    }
                }
            }
            // positions sort into owner groups (shards own ascending ranges)
            std::sort(hpos.begin(), hpos.end());
            auto& hl = h->halo[s];
            hl.resize(hpos.size());
            auto& g = h->group[s];
            g.assign(S + 1, 0);
            for (size_t j = 0; j < hpos.size(); ++j) {
                hl[j] = src->order[hpos[j]];
                slot[hpos[j]] = n_own + (int64_t)j;
                g[src->owner[hl[j]] + 1]++;
            }
            for (int q = 0; q < S; ++q) g[q + 1] += g[q];
            if (n_own + (int64_t)hpos.size() > INT32_MAX) {
                delete h;
                return mfd::fail(MFD_ERR_ARG, "mfd_halo_create: a shard's local array exceeds int32 indexing");
            }
            for (int k = 0; k < nsets; ++k) {
                const mfd_partition* c = centres[k];
                const int64_t a = c->start[s], b = c->start[s + 1];
                auto& L = h->local[k][s];
                L.resize((b - a) * (int64_t)ncols[k]);
                for (int64_t r = a; r < b; ++r) {
                    const int64_t* row = idx[k] + c->order[r] * (int64_t)ncols[k];
                    for (int j = 0; j < ncols[k]; ++j) {
                        int64_t p = src->pos[row[j]];
                        int64_t li = (p >= own_a && p < own_b) ? p - own_a : slot[p];
                        L[(r - a) * ncols[k] + j] = (int32_t)li;
                    }
                }
            }
        }
        *out = h;
        return MFD_OK;
    } catch (const std::bad_alloc&) {
        return mfd::fail(MFD_ERR_OOM, "mfd_halo_create: host allocation failed");
    }
}

mfd_status mfd_halo_nodes(const mfd_halo* halo, int shard, int64_t* count, int64_t* ids) {
    if (!halo || !count || shard < 0 || shard >= halo->nshards)
        return mfd::fail(MFD_ERR_ARG, "mfd_halo_nodes: null plan, null count or bad shard");
    const auto& hl = halo->halo[shard];
    *count = (int64_t)hl.size();
    if (ids && !hl.empty()) std::memcpy(ids, hl.data(), sizeof(int64_t) * hl.size());
    return MFD_OK;
}

mfd_status mfd_halo_send(const mfd_halo* halo, int from, int to, int64_t* count, int64_t* ids) {
    if (!halo || !count || from < 0 || to < 0 || from >= halo->nshards || to >= halo->nshards)
        return mfd::fail(MFD_ERR_ARG, "mfd_halo_send: null plan, null count or bad shard");
    const auto& g = halo->group[to];
    const int64_t a = g[from], b = g[from + 1];
    *count = b - a;
    if (ids)
        for (int64_t j = a; j < b; ++j) ids[j - a] = halo->halo[to][j];
    return MFD_OK;
}

mfd_status mfd_halo_local_idx(const mfd_halo* halo, int shard, int set, int32_t* local_idx) {
    if (!halo || shard < 0 || shard >= halo->nshards || set < 0 || set >= halo->nsets)
        return mfd::fail(MFD_ERR_ARG, "mfd_halo_local_idx: null plan, bad shard or bad set");
    const auto& L = halo->local[set][shard];
    if (!L.empty()) {
        if (!local_idx) return mfd::fail(MFD_ERR_ARG, "mfd_halo_local_idx: local_idx is null");
        std::memcpy(local_idx, L.data(), sizeof(int32_t) * L.size());
    }
    return MFD_OK;
}

void mfd_halo_destroy(mfd_halo* halo) { delete halo; }

}  // extern "C"
