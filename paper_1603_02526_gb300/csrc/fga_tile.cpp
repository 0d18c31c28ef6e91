// fga_tile.cpp -- host planner of the disk-tile sweep (see tile_internal.h).
//
// Input: the disk pairs, walls and radius rewards of a packing graph.
// Output: the units (32 row disks x 8 column disks of the pair matrix) in
// blocks of row blocks x column groups, their assignment to CTAs (one unit per warp, or several
// per warp on larger graphs), each CTA's
// z table (slots = disks it touches), the staging positions of every
// contribution to a slot variable and the order they are summed in, and
// the CTA that owns each variable (writes its z, adds its dual residual and
// clears its accumulator for reuse).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "tile_internal.h"

namespace fga {

int tile_plan(const TileInput &in, TilePlan &P, std::string &why) {
    const int64_t npairs = (int64_t)in.c1.size();
    if (npairs == 0) {
        why = "no disk pairs";
        return 1;
    }
    if (in.sms <= 0 || in.wmax <= 0) {
        why = "no launch shape";
        return 1;
    }
    // 1. disks: a centre variable and a radius variable, consistently paired
    std::unordered_map<int32_t, int32_t> c2r, r2c;
    auto add_disk = [&](int32_t c, int32_t r) -> bool {
        auto a = c2r.find(c);
        if (a != c2r.end() && a->second != r) return false;
        auto b = r2c.find(r);
        if (b != r2c.end() && b->second != c) return false;
        c2r[c] = r;
        r2c[r] = c;
        return true;
    };
    for (int64_t p = 0; p < npairs; ++p) {
        if (!add_disk(in.c1[p], in.r1[p]) || !add_disk(in.c2[p], in.r2[p])) {
            why = "a centre variable appears with two radius variables";
            return 1;
        }
    }
    for (const auto &L : in.locs) {
        if (L.c >= 0) {
            if (!add_disk(L.c, L.r)) {
                why = "a wall pairs a centre with another radius";
                return 1;
            }
        } else if (!r2c.count(L.r)) {
            why = "a radius reward on a variable that is no disk radius";
            return 1;
        }
    }
    std::vector<int32_t> centres;
    centres.reserve(c2r.size());
    for (const auto &kv : c2r) centres.push_back(kv.first);
    std::sort(centres.begin(), centres.end());
    const int64_t ND = (int64_t)centres.size();
    std::unordered_map<int32_t, int32_t> disk_of_c;
    for (int64_t d = 0; d < ND; ++d) disk_of_c[centres[d]] = (int32_t)d;
    std::vector<int32_t> disk_r((size_t)ND);
    for (int64_t d = 0; d < ND; ++d) disk_r[d] = c2r[centres[d]];

    // 2. units: (row block, column group, layer); a duplicate pair goes to
    // the next layer of its (row block, column group)
    const int64_t NJ = (ND + kTileCols - 1) / kTileCols;
    struct UnitTmp {
        int64_t I, J;
        int layer;
        uint8_t m[kTileRows];
    };
    std::vector<UnitTmp> ut;
    std::unordered_map<int64_t, std::vector<int32_t>> layers;   // key I * NJ + J -> unit ids by layer
    std::vector<int32_t> tmp_pos((size_t)npairs);
    for (int64_t p = 0; p < npairs; ++p) {
        const int64_t a = disk_of_c[in.c1[p]], b = disk_of_c[in.c2[p]];
        const int64_t I = a / kTileRows, J = b / kTileCols;
        const int l = (int)(a % kTileRows), c = (int)(b % kTileCols);
        auto &ls = layers[I * NJ + J];
        int32_t uid = -1;
        for (int32_t k : ls)
            if (!((ut[k].m[l] >> c) & 1u)) { uid = k; break; }
        if (uid < 0) {
            UnitTmp t;
            t.I = I;
            t.J = J;
            t.layer = (int)ls.size();
            std::memset(t.m, 0, sizeof t.m);
            uid = (int32_t)ut.size();
            ut.push_back(t);
            ls.push_back(uid);
        }
        ut[uid].m[l] |= (uint8_t)(1u << c);
        // lane l keeps column c in register slot c ^ ((l >> 2) & 7): with
        // this relabelling the kernel's reduce-scatter over the lanes needs
        // no selects
        tmp_pos[p] = uid * 256 + (c ^ ((l >> 2) & 7)) * 32 + l;
    }
    const int64_t U = (int64_t)ut.size();
    // sparse pair sets would waste most lanes; a graph of at most one unit
    // per SM runs in one wave whatever its fill
    if (U > in.sms && (double)npairs < 0.5 * 256.0 * (double)U) {
        why = "disk pairs fill less than half of their tiles";
        return 1;
    }
    // CTAs take W consecutive units of this order.  When a CTA has more
    // units than warps, units are grouped in blocks of GR row blocks x GC
    // column groups (row-major inside a block): W units of one block touch
    // about 32 GR + 8 GC disks, against 32 + 8 W for W units of one row
    // block, so the CTA's z tables and count-and-sum contributions are
    // fewer (GR ~ sqrt(W / 4) minimises 32 GR + 8 W / GR; measured: N = 2500
    // from 16.6 to 14.9 us per iteration, its tables from 212 to 183 KB).
    // With one unit per warp, row-major order (GR = 1) measured faster
    // (N = 1000: 2.99 against 3.47 us).  The choice depends on the graph
    // only (the kernel's most warps per CTA), not on a smaller block asked
    // for with FGA_OPT_BLOCK, so that such a block runs the same plan.
    const int64_t W0 = std::max<int64_t>(1, (U + in.sms - 1) / in.sms);
    const int64_t GR =
        W0 <= kTileMaxWarps ? 1 : std::max<int64_t>(1, (int64_t)std::llround(std::sqrt((double)W0 / 4.0)));
    const int64_t GC = std::max<int64_t>(1, (W0 + GR - 1) / GR);
    std::vector<int32_t> order((size_t)U), rank((size_t)U);
    for (int64_t i = 0; i < U; ++i) order[i] = (int32_t)i;
    std::sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        const int64_t bx = ut[x].I / GR, by = ut[y].I / GR;
        if (bx != by) return bx < by;
        const int64_t cx = ut[x].J / GC, cy = ut[y].J / GC;
        if (cx != cy) return cx < cy;
        if (ut[x].I != ut[y].I) return ut[x].I < ut[y].I;
        if (ut[x].J != ut[y].J) return ut[x].J < ut[y].J;
        return ut[x].layer < ut[y].layer;
    });
    for (int64_t i = 0; i < U; ++i) rank[order[i]] = (int32_t)i;
    P.pair_pos.resize((size_t)npairs);
    for (int64_t p = 0; p < npairs; ++p) P.pair_pos[p] = rank[tmp_pos[p] / 256] * 256 + tmp_pos[p] % 256;

    // 3. launch shape: as few units per CTA as fit the SMs, one warp each up
    // to the kernel's warps per CTA; beyond that each warp takes several in
    // turn (their state then lives in device memory between passes)
    const int64_t W = (U + in.sms - 1) / in.sms;
    if (W > kTileMaxUnitsMulti) {
        why = "more units per CTA than the tables of one CTA can hold";
        return 1;
    }
    if (U * (int64_t)kUnitEdges > (int64_t)INT32_MAX / 2) {
        why = "too many units";
        return 1;
    }
    const int G = (int)((U + W - 1) / W);
    P.U = (int)U;
    P.W = (int)W;
    P.G = G;
    P.warps = (int)std::min<int64_t>(W, in.wmax);

    // 4. per CTA: slots (disks) of its units
    P.rowslot.assign((size_t)U * kTileRows, 0);
    P.colslot.assign((size_t)U * kTileCols, 0);
    P.mask.assign((size_t)U * kTileRows, 0);
    std::vector<std::vector<int32_t>> slots((size_t)G);           // disk of each slot
    std::vector<int32_t> stamp((size_t)ND, -1), slot_of((size_t)ND, 0);
    std::vector<std::vector<int32_t>> disk_ctas((size_t)ND);      // CTAs that hold the disk
    auto slot_for = [&](int g, int32_t d) {
        if (stamp[d] != g) {
            stamp[d] = g;
            slot_of[d] = (int32_t)slots[g].size();
            slots[g].push_back(d);
            disk_ctas[d].push_back(g);
        }
        return slot_of[d];
    };
    for (int g = 0; g < G; ++g) {
        const int64_t u0 = (int64_t)g * W, u1 = std::min<int64_t>(U, u0 + W);
        for (int64_t r = u0; r < u1; ++r) {
            const UnitTmp &t = ut[order[r]];
            uint8_t colany = 0;
            for (int l = 0; l < kTileRows; ++l) colany |= t.m[l];
            for (int l = 0; l < kTileRows; ++l) {
                uint8_t mp = 0;   // bit j: pair of register slot j (column j ^ ((l >> 2) & 7))
                for (int j = 0; j < kTileCols; ++j)
                    if ((t.m[l] >> (j ^ ((l >> 2) & 7))) & 1u) mp |= (uint8_t)(1u << j);
                P.mask[r * kTileRows + l] = mp;
                if (t.m[l]) P.rowslot[r * kTileRows + l] = (uint16_t)slot_for(g, (int32_t)(t.I * kTileRows + l));
            }
            for (int c = 0; c < kTileCols; ++c)
                if ((colany >> c) & 1u) P.colslot[r * kTileCols + c] = (uint16_t)slot_for(g, (int32_t)(t.J * kTileCols + c));
        }
    }
    // 5. walls and radius rewards: to the CTA holding their disk with the
    // fewest such factors so far (disks of no unit make the graph unsuitable)
    std::vector<std::vector<int32_t>> cta_locs((size_t)G);
    for (int32_t i = 0; i < (int32_t)in.locs.size(); ++i) {
        const auto &L = in.locs[i];
        const int32_t d = disk_of_c[L.c >= 0 ? L.c : r2c[L.r]];
        if (disk_ctas[d].empty()) {
            why = "a wall or reward on a disk without pairs";
            return 1;
        }
        int best = disk_ctas[d][0];
        for (int g : disk_ctas[d])
            if (cta_locs[g].size() < cta_locs[best].size()) best = g;
        cta_locs[best].push_back(i);
    }
    for (int g = 0; g < G; ++g) {
        if (slots[g].size() > 65535) {
            why = "a CTA touches more than 65535 disks";
            return 1;
        }
    }

    // 6. slot-vars, their contributions, and the variable-major partials
    P.cta.resize((size_t)G);
    P.sv.clear();
    P.zden.clear();
    P.cptr.assign(1, 0);
    P.clist.clear();
    P.loc.clear();
    P.loc_member.clear();
    P.loc_bucket_type.clear();
    std::vector<int64_t> pcount((size_t)in.nz, 0);
    int smax = 1, stgmax = 1, svmax = 3, locmax = 1, clmax = 1;
    for (int g = 0; g < G; ++g) {
        const int64_t u0 = (int64_t)g * W, u1 = std::min<int64_t>(U, u0 + W);
        TileCta &C = P.cta[g];
        std::memset(&C, 0, sizeof C);
        C.unit0 = (int)u0;
        C.nunit = (int)(u1 - u0);
        C.sv0 = (int)P.sv.size();
        const int ns = (int)slots[g].size();
        C.nsv = 3 * ns;
        C.loc0 = (int)P.loc.size();
        C.nloc = (int)cta_locs[g].size();
        for (int s = 0; s < ns; ++s) slot_of[slots[g][s]] = s;
        std::vector<std::vector<int32_t>> contrib((size_t)3 * ns);
        for (int64_t r = u0; r < u1; ++r) {
            const int w = (int)(r - u0);
            const UnitTmp &t = ut[order[r]];
            uint8_t colany = 0;
            for (int l = 0; l < kTileRows; ++l) colany |= t.m[l];
            for (int l = 0; l < kTileRows; ++l) {
                if (!t.m[l]) continue;
                const int s = slot_of[t.I * kTileRows + l];
                for (int q = 0; q < 3; ++q) contrib[3 * s + q].push_back(w * kUnitStage + q * kTileRows + l);
            }
            for (int c = 0; c < kTileCols; ++c) {
                if (!((colany >> c) & 1u)) continue;
                const int s = slot_of[t.J * kTileCols + c];
                for (int q = 0; q < 3; ++q)
                    contrib[3 * s + q].push_back(w * kUnitStage + 3 * kTileRows + q * kTileCols + c);
            }
        }
        int stg = C.nunit * kUnitStage;
        for (int32_t i : cta_locs[g]) {
            const auto &L = in.locs[i];
            const int32_t d = disk_of_c[L.c >= 0 ? L.c : r2c[L.r]];
            const int s = slot_of[d];
            TileLocal tl;
            std::memset(&tl, 0, sizeof tl);
            tl.type = L.type;
            tl.slot = s;
            tl.stg = stg;
            for (int k = 0; k < 5; ++k) tl.p[k] = L.p[k];
            if (L.c >= 0) {
                for (int q = 0; q < 3; ++q) contrib[3 * s + q].push_back(stg + q);
                stg += 3;
            } else {
                contrib[3 * s + 2].push_back(stg);
                stg += 1;
            }
            P.loc.push_back(tl);
            P.loc_member.push_back(L.member);
            P.loc_bucket_type.push_back(L.type);
        }
        for (int s = 0; s < ns; ++s) {
            const int32_t d = slots[g][s];
            const int32_t vars[3] = {centres[d], centres[d] + 1, disk_r[d]};
            for (int q = 0; q < 3; ++q) {
                const int32_t v = vars[q];
                // .y/.z (the variable's partial row) are set below; .w holds
                // this CTA's index inside the row for now
                P.sv.push_back(make_int4(v, 0, 0, (int)pcount[v]));
                pcount[v]++;
                P.zden.push_back((float)in.deg[v]);
                for (int32_t j : contrib[3 * s + q]) P.clist.push_back(j);
                P.cptr.push_back((int32_t)P.clist.size());
            }
        }
        smax = std::max(smax, ns);
        stgmax = std::max(stgmax, stg);
        svmax = std::max(svmax, C.nsv);
        locmax = std::max(locmax, C.nloc);
        clmax = std::max(clmax, P.cptr.back() - P.cptr[C.sv0]);
    }
    // one fixed-point accumulator per variable; the owner of a variable is
    // its first holder
    for (int64_t v = 0; v < in.nz; ++v) {
        if (pcount[v] > kTileMaxHolders) {
            why = "a variable is held by too many CTAs";
            return 1;
        }
    }
    for (int4 &d : P.sv) {
        const int k = d.w;
        d.y = (int)pcount[d.x];
        d.z = 0;
        d.w = k == 0 ? (int)0x80000000u : 0;
    }
    if (stgmax > 65535) {
        why = "a CTA stages more than 2^16 values";
        return 1;
    }
    P.ptot = (int)std::max<int64_t>(in.nz, 1);
    P.smax = smax;
    P.stgmax = stgmax;
    P.svmax = svmax;
    P.locmax = locmax;
    P.clmax = clmax;
    // every variable of a disk must be gathered somewhere
    for (int64_t d = 0; d < ND; ++d) {
        if (pcount[centres[d]] == 0 || pcount[disk_r[d]] == 0) {
            why = "a disk with no unit";
            return 1;
        }
    }
    return 0;
}

}  // namespace fga
