// Test driver (host only): runs the disk-tile planner on the circle-packing
// graph of N disks and writes the plan's tables to files, for
// tests/test_tile_plan_host.py to check.
//
// The graph is built as paper_1603_02526_gb300.inputs.packing_problem
// builds it: disk i has its centre at scalar variables 3i, 3i + 1 and its
// radius at 3i + 2; the pairs (i < j) in row-major order, then three walls
// per disk, then one linear radius reward per disk.
//
// usage: tile_plan_check N SMS WMAX OUTDIR
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "tile_internal.h"

template <typename T>
static void dump(const std::string &dir, const char *name, const std::vector<T> &v) {
    const std::string path = dir + "/" + name;
    FILE *f = std::fopen(path.c_str(), "wb");
    if (!f) std::exit(3);
    if (!v.empty() && std::fwrite(v.data(), sizeof(T), v.size(), f) != v.size()) std::exit(3);
    std::fclose(f);
}

int main(int argc, char **argv) {
    if (argc != 5) return 2;
    const int N = std::atoi(argv[1]);
    const std::string dir = argv[4];
    fga::TileInput in;
    in.nz = 3 * (int64_t)N;
    in.sms = std::atoi(argv[2]);
    in.wmax = std::atoi(argv[3]);
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            in.c1.push_back(3 * i);
            in.r1.push_back(3 * i + 2);
            in.c2.push_back(3 * j);
            in.r2.push_back(3 * j + 2);
        }
    int64_t member = 0;
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < 3; ++k) {
            fga::TileInput::Local L{};
            L.type = 1;   // wall
            L.c = 3 * i;
            L.r = 3 * i + 2;
            L.member = member++;
            in.locs.push_back(L);
        }
    for (int i = 0; i < N; ++i) {
        fga::TileInput::Local L{};
        L.type = 2;   // linear radius reward
        L.c = -1;
        L.r = 3 * i + 2;
        L.member = i;
        in.locs.push_back(L);
    }
    in.deg.assign((size_t)in.nz, 0.0);
    for (int i = 0; i < N; ++i) {
        in.deg[3 * i] = in.deg[3 * i + 1] = (N - 1) + 3;
        in.deg[3 * i + 2] = (N - 1) + 3 + 1;
    }

    fga::TilePlan P;
    std::string why;
    const int rc = fga::tile_plan(in, P, why);
    const fga::TileSmem L = fga::tile_smem_layout(P.smax, P.svmax, P.locmax, P.clmax, P.stgmax);
    {
        const std::string path = dir + "/meta.txt";
        FILE *f = std::fopen(path.c_str(), "w");
        if (!f) return 3;
        std::fprintf(f, "rc %d\nU %d\nW %d\nG %d\nwarps %d\nptot %d\nsmax %d\nstgmax %d\nsvmax %d\nlocmax %d\n"
                        "clmax %d\nsmem %d\nnpairs %zu\n",
                     rc, P.U, P.W, P.G, P.warps, P.ptot, P.smax, P.stgmax, P.svmax, P.locmax, P.clmax, L.total,
                     in.c1.size());
        std::fprintf(f, "why %s\n", why.empty() ? "-" : why.c_str());
        std::fclose(f);
    }
    if (rc) return 0;
    std::vector<int32_t> cta, sv, loc;
    for (const auto &C : P.cta) {
        const int32_t row[6] = {C.unit0, C.nunit, C.sv0, C.nsv, C.loc0, C.nloc};
        cta.insert(cta.end(), row, row + 6);
    }
    for (const auto &d : P.sv) {
        const int32_t row[4] = {d.x, d.y, d.z, d.w};
        sv.insert(sv.end(), row, row + 4);
    }
    for (const auto &l : P.loc) {
        const int32_t row[3] = {l.type, l.slot, l.stg};
        loc.insert(loc.end(), row, row + 3);
    }
    dump(dir, "pair_pos.i32", P.pair_pos);
    dump(dir, "rowslot.u16", P.rowslot);
    dump(dir, "colslot.u16", P.colslot);
    dump(dir, "mask.u8", P.mask);
    dump(dir, "cta.i32", cta);
    dump(dir, "sv.i32", sv);
    dump(dir, "zden.f32", P.zden);
    dump(dir, "cptr.i32", P.cptr);
    dump(dir, "clist.i32", P.clist);
    dump(dir, "loc.i32", loc);
    dump(dir, "loc_member.i64", P.loc_member);
    dump(dir, "loc_type.i32", P.loc_bucket_type);
    return 0;
}
