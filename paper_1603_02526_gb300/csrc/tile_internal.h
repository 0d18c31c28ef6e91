// tile_internal.h -- the disk-tile sweep: descriptors shared by the host
// planner (fga_tile.cpp) and the kernel (sweep_tile.cu).  Not part of the
// public C-ABI.
//
// A graph qualifies when it holds only circle-packing factors (disk pairs,
// walls, radius rewards), runs in FP32 with one rho and one alpha, and its
// disk pairs fill most of a 32 x 8 tiling of the pair matrix.  Disks are
// numbered by the scalar id of their centre.  A disk pair (a, b) sits in
// unit (a / 32, b / 8) at lane l = a % 32 and column c = b % 8, which the
// lane keeps in register slot c ^ ((l >> 2) & 7); a warp owns one unit for
// the whole call and keeps the unit's 1,536 u values in registers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "fga_internal.h"

namespace fga {

constexpr int kTileRows = 32;                               // disks per row block (one per lane)
constexpr int kTileCols = 8;                                // disks per column group
constexpr int kUnitEdges = kTileRows * kTileCols * 6;       // storage slots of one unit
constexpr int kUnitStage = 3 * kTileRows + 3 * kTileCols;   // staged partial sums of one unit
constexpr int kTileMaxWarps = 16;                           // warps per CTA, at most
constexpr int kTileMaxUnitsMulti = 256;                     // units per CTA, at most (several per warp)
constexpr int kTileMaxHolders = 255;                        // CTAs holding one variable, at most
// Per-CTA partial sums are added into one 64-bit word per variable: the
// count of contributions in the top 8 bits (2^56 per contribution, modulo
// 256) and the sum in fixed point (scale 2^32) below, both by one integer
// addition of 2^56 + q.  Integer addition is exact and associative, so the
// sum does not depend on the order in which the CTAs' additions land, and a
// reader knows from the word alone when every holder has added.  Two words
// per variable: pass p adds into word p mod 2, pass p + 1 reads it.  A word
// only grows (it is never cleared during a launch), and a CTA reads each
// variable's new contributions as the difference to the word it saw two
// passes before, complete when that difference counts the variable's
// holders.  No contribution of a later pass can be in it yet: a holder adds
// to the same word again only in pass p + 2, after its own pass p + 1
// gather, which waits for this CTA's pass p + 1 contribution to the same
// variable, made after this read.
// A partial of magnitude 2^14 or more (or not finite) is reported as a
// non-finite residual; with at most kTileMaxHolders partials one pass's sum
// stays below 2^54 in magnitude, clear of the count bits.
constexpr float kTileFixScale = 4294967296.0f;              // 2^32
constexpr float kTileFixInv = 2.3283064365386963e-10f;      // 2^-32
constexpr float kTileFixMax = 16384.0f;                     // 2^14
constexpr unsigned long long kTileCountUnit = 1ull << 56;

// A wall or radius factor, processed by one thread of the CTA it is given
// to.  p: wall Qx, Qy, Vx, Vy, 1 / (|Q|^2 + 1); linear reward w / rho;
// area reward 1 / (rho - 1).
struct TileLocal {
    int type;   // FGA_PACK_WALL (3 edges) or FGA_PACK_RADIUS_LIN / _QUAD (1 edge)
    int e0;     // storage index of the first edge
    int slot;   // the disk's slot in the CTA's z table
    int stg;    // first staging position
    float p[5];
    int pad[3];
};

// Per CTA: its units (one per warp), its scalar variables ("slot-vars",
// three per slot: centre x, centre y, radius), its local factors.
struct TileCta {
    int unit0, nunit;
    int sv0, nsv;
    int loc0, nloc;
    int pad[2];
};

// Barrier word of the tile kernel: a counter that only grows (arrivals of
// all CTAs over all iterations of a launch) and the error word, at the same
// offset as Barrier::error so that the host reads both the same way.
struct TileSync {
    unsigned long long count;
    int error;
    int overflow;   // a partial sum out of the fixed-point range
};
static_assert(sizeof(TileSync) == sizeof(Barrier), "TileSync and Barrier share one buffer");
static_assert(offsetof(TileSync, error) == offsetof(Barrier, error), "error words must coincide");

// Shared memory of one CTA (byte offsets, each 16-byte aligned): z, the
// previous z, y = 2 z - z_prev and the previous y per slot (float4: x, y,
// r, unused), slot-var descriptors, the
// walls and rewards with their u, the edge counts, the contribution lists,
// and the staging area of the partial sums.
struct TileSmem {
    int z4, zp4, y4, yp4, sv, loc, uloc, zden, cptr, clist, stg, pv, total;
};
inline __host__ __device__ constexpr int tile_align16(int v) { return (v + 15) & ~15; }
inline __host__ __device__ TileSmem tile_smem_layout(int smax, int svmax, int locmax, int clmax, int stgmax) {
    TileSmem L{};
    int o = 0;
    L.z4 = o;
    o = tile_align16(o + smax * 16);
    L.zp4 = o;
    o = tile_align16(o + smax * 16);
    L.y4 = o;
    o = tile_align16(o + smax * 16);
    L.yp4 = o;
    o = tile_align16(o + smax * 16);
    L.sv = o;
    o = tile_align16(o + svmax * 16);
    L.loc = o;
    o = tile_align16(o + locmax * (int)sizeof(TileLocal));
    L.uloc = o;
    o = tile_align16(o + locmax * 32);
    L.zden = o;
    o = tile_align16(o + svmax * 4);
    L.cptr = o;
    o = tile_align16(o + (svmax + 1) * 4);
    L.clist = o;   // 16-bit staging positions (the planner keeps the staging area below 2^16 values)
    o = tile_align16(o + clmax * 2);
    L.stg = o;
    o = tile_align16(o + stgmax * 4);
    L.pv = o;   // per slot-var and word: the value seen the last time
    o = tile_align16(o + svmax * 16);
    L.total = o;
    return L;
}

struct TileArgs {
    int G;          // CTAs
    int U;          // units
    int smax;       // slots of the largest z table
    int stgmax;     // staging floats of the largest CTA
    int svmax;      // slot-vars of the largest CTA
    int locmax;     // walls and rewards of the largest CTA
    int clmax;      // contributions of the largest CTA
    const TileCta *cta;
    const unsigned short *rowslot;   // [U][32] slot of each lane's row disk
    const unsigned short *colslot;   // [U][8]  slot of each column disk
    const unsigned char *mask;       // [U][32] bit j: the pair of register slot j exists
    const int4 *sv;                  // per slot-var: var, holders, unused, owner << 31
    const float *zden;               // per slot-var: number of edges of the variable
    const int *cptr;                 // per slot-var: contributions cptr[i] .. cptr[i + 1] in clist
    const int *clist;                // staging positions (relative to the CTA's staging area)
    const TileLocal *loc;
    const double *srho2;             // per variable: sum of rho^2 over its edges
    float *u;                        // per edge (storage order)
    float *dsave;                    // alpha = 1: [U][24][32] displacements kept for the next check
    float *dres;                     // alpha = 1: [U][24][32] displacements of the stored state
    float *dlive;                    // more units than warps per CTA: [U][24][32] the live
                                     // displacements (alpha = 1) between a unit's turns; null when
                                     // every unit has its own warp (state in registers)
    float *lres;                     // alpha = 1: per wall / reward, its displacement parameter
                                     // of the stored state
    const float *zpin;               // alpha = 1: z before the stored state (resume)
    float *zpout;                    // alpha = 1: written at checks with the state
    int resume;                      // alpha = 1: dres / zpin hold the state this call starts from
    float *xout;                     // x buffer written at checks and at the end
    const float *zin;                // z at the start of the call
    float *zout;                     // z written at checks and at the end
    unsigned long long *acc;         // [2][ptot] count and fixed-point sum per variable (see
                                     // kTileCountUnit), zeroed before a launch
    int ptot;                        // scalar variables
    double *res;                     // [2][2][G] residual partial sums (pri, dual)
    int pair_ebase;                  // storage index of unit 0
    float alpha;
    long long E;
    Ctl *ctl;
    TileSync *sync;
    long long k0, K;
    int check_every;
    double tol_pri, tol_dual;
    long long timeout_ns;
    int skip_block;
    int xw, zw;                      // buffers written (for the control block)
};

// Host planner input: the graph's packing factors in bucket order.
struct TileInput {
    int64_t nz = 0;
    // disk pairs: scalar ids of the two centres (first coordinate) and radii
    std::vector<int32_t> c1, r1, c2, r2;
    // walls (c, r, Q, V) and radius rewards (r, parameter)
    struct Local {
        int type;
        int32_t c, r;          // c = -1 for a radius reward
        int64_t member;        // factor index inside its bucket
        float p[5];
    };
    std::vector<Local> locs;
    std::vector<double> deg;   // per scalar variable: number of edges
    int sms = 0;
    int wmax = 0;              // warps per CTA the kernel can run with
};

struct TilePlan {
    int U = 0, W = 0, G = 0, smax = 0, stgmax = 0, svmax = 0, locmax = 0, clmax = 0;
    int warps = 0;                      // warps per CTA: W when W <= the kernel's warps, else that
                                        // maximum (each warp then takes several units in turn)
    int ptot = 0;                       // accumulators per buffer (scalar variables)
    std::vector<int32_t> pair_pos;      // per disk pair (bucket order): unit * 256 + slot * 32 + lane
    std::vector<TileCta> cta;
    std::vector<uint16_t> rowslot, colslot;
    std::vector<uint8_t> mask;
    std::vector<int4> sv;
    std::vector<float> zden;
    std::vector<int32_t> cptr, clist;
    std::vector<TileLocal> loc;         // e0 filled in after the storage layout
    std::vector<int64_t> loc_member;    // bucket member of each local item (same order as loc)
    std::vector<int> loc_bucket_type;   // its type
};

// Builds the plan; returns 0 when the graph qualifies, 1 (reason in `why`)
// when it does not.
int tile_plan(const TileInput &in, TilePlan &P, std::string &why);

// Kernel launch (sweep_tile.cu) and the warps per CTA it can run with.
cudaError_t tile_sweep_launch(const TileArgs &a, int block, int smem, cudaStream_t s);
// The latency floor of a pass on the same grid (mode 0: barrier; 1: gather
// loads, accumulator reductions and barrier), `iters` passes.
cudaError_t tile_floor_launch(const TileArgs &a, long long iters, int mode, int block, int smem, cudaStream_t s);
int tile_max_warps();
int tile_smem_bytes(const TilePlan &P);

}  // namespace fga
