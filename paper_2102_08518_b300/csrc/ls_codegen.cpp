// Code generator: sub-region table -> specialised CUDA C++ (Sec. 4).
//
// The paper composes "blocks" (preamble, coset loop, region of evaluation,
// sub-region membership, table lookups, reference sub-region loop, polynomial
// evaluation) into LLVM-IR.  This generator composes the same blocks into CUDA
// C++ that NVRTC compiles for sm_103a:
//   * region of evaluation: floor (parallelepiped) or nearest site per coset
//     (Voronoi), branch-free selects;
//   * sub-region membership: signed-permutation folding (|y| sorted by a
//     3-element network gives T of Algorithm 1 without a table) followed by the
//     BSP plane tests + sigma LUT among the reference sub-regions;
//   * memory lookup: one array per Cartesian coset, addresses built from
//     per-point coset bases and reference-axis strides, the whole stencil
//     unrolled with every offset an immediate; a bounds-checked copy of the
//     gathers is taken only by points whose stencil leaves the arrays;
//   * polynomial evaluation: the site coefficients are folded into the
//     monomial coefficients A_a = sum_j M[j][a] c_j (M baked in as FP32
//     immediates), then one multivariate Horner form per reference sub-region;
//     tensor-product splines use per-axis Horner weights and a nested
//     contraction instead.
#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <functional>
#include <map>
#include <set>
#include <sstream>

#include "ls_internal.h"

namespace ls {
namespace {

std::string flit(double v)
{
    float f = (float)v;
    if (f == 0.0f) return "0.0f";
    char buf[64];
    std::snprintf(buf, sizeof buf, "%af", (double)f);
    return buf;
}

struct Emitter {
    std::ostringstream o;
    int tmp = 0;
    int fma = 0;
    std::string ld = "ls_ld_f32";     // coefficient loader of the spline being emitted
    bool brick = false;               // bricked coefficient layout (else linear)
    bool sym = true;                  // factored coefficient transform (butterflies + sparser M)
    bool brick_shift = false;         // shifted bricked copies (LS_LAYOUT_BRICKED_SHIFTED[_XYZ])
    int shift_axes = 2;               // axes the copies shift (2: four copies, 3: eight)
    unsigned long long shift_mask[3] = {0, 0, 0};   // their copy-choice rule (shift_rule)
    int wait_rounds = 1 << 20;        // try_wait rounds of a bounded wait (ls_mbar_wait; polls: x4)
    bool no_signal = false;           // test hook: warp-specialized producers never signal their slots
    bool l2_keep = false;             // coefficient loads carry an L2 evict-last cache policy
    bool fma2 = false;                // factored transform in paired FP32 FMA (fma.rn.f32x2)
    std::string ktabs;                // __constant__ tables of the paired transform's constant pairs
    std::map<std::string, std::string> kname_of;   // table text -> its name (shared by the kernels)
    std::string fresh(const char *p) { return std::string(p) + std::to_string(tmp++); }
};

// Union of site lists in first-seen order; index maps per region.
struct Stencil {
    std::vector<I3> sites;
    std::vector<std::vector<int>> region_to_union;
};

Stencil union_stencil(const Table &t)
{
    Stencil s;
    std::map<I3, int> idx;
    for (const auto &r : t.ref) {
        std::vector<int> m;
        for (const auto &site : r.sites) {
            auto it = idx.find(site);
            if (it == idx.end()) {
                idx[site] = (int)s.sites.size();
                m.push_back((int)s.sites.size());
                s.sites.push_back(site);
            } else {
                m.push_back(it->second);
            }
        }
        s.region_to_union.push_back(m);
    }
    return s;
}

int floordiv2(int v) { return (v >= 0) ? v / 2 : -((-v + 1) / 2); }

// ---------------------------------------------------------------------------
// common prologue: helpers and argument structs
// ---------------------------------------------------------------------------
const char *loader_name(ls_dtype dt)
{
    return dt == LS_BF16 ? "ls_ld_bf16" : dt == LS_F16 ? "ls_ld_f16" : "ls_ld_f32";
}

void emit_prologue(Emitter &e)
{
    auto &o = e.o;
    o << "// generated by the lattice spline code generator; do not edit\n";
    o << "typedef unsigned short ls_u16;\n";
    if (e.l2_keep) {
        // coefficient loads with an L2 evict-last policy: the volume's lines
        // outlast the evict-first point and result streams (the policy is a
        // pure value: one createpolicy per kernel after common-subexpression
        // elimination)
        o << "static __device__ __forceinline__ unsigned long long ls_keep_pol() { unsigned long long q;"
             " asm(\"createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\" : \"=l\"(q)); return q; }\n";
        o << "static __device__ __forceinline__ float ls_ldk_f32(const float* p) { float v;"
             " asm(\"ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;\" : \"=f\"(v) : \"l\"(p), \"l\"(ls_keep_pol()));"
             " return v; }\n";
        o << "static __device__ __forceinline__ ls_u16 ls_ldk_u16(const ls_u16* p) { ls_u16 v;"
             " asm(\"ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;\" : \"=h\"(v) : \"l\"(p), \"l\"(ls_keep_pol()));"
             " return v; }\n";
        o << "static __device__ __forceinline__ float ls_ld_f32(const void* p, int i) {"
             " return ls_ldk_f32((const float*)p + i); }\n";
        o << "static __device__ __forceinline__ float ls_ld_bf16(const void* p, int i) {"
             " return __uint_as_float(((unsigned)ls_ldk_u16((const ls_u16*)p + i)) << 16); }\n";
    } else {
        o << "static __device__ __forceinline__ float ls_ld_f32(const void* p, int i) {"
             " return __ldg((const float*)p + i); }\n";
        o << "static __device__ __forceinline__ float ls_ld_bf16(const void* p, int i) {"
             " return __uint_as_float(((unsigned)__ldg((const ls_u16*)p + i)) << 16); }\n";
    }
    o << "static __device__ __forceinline__ float ls_sh_ld(const void* p, int i) { return ((const float*)p)[i]; }\n";
    // point coordinates and results stream through once: evict-first in L1 and
    // L2 (ld/st .cs), so that the coefficient lines stay resident in L2
    o << "static __device__ __forceinline__ float ls_ld_pt(const float* p) { return __ldcs(p); }\n";
    o << "static __device__ __forceinline__ void ls_st_out(float* p, float v) { __stcs(p, v); }\n";
    // one 32-byte load (a whole sector) into eight floats: p must be 32-byte aligned
    o << "static __device__ __forceinline__ void ls_ld8(const float* p, float& r0, float& r1, float& r2, float& r3,"
         " float& r4, float& r5, float& r6, float& r7) { asm(\"ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6,"
         " %7}, [%8];\" : \"=f\"(r0), \"=f\"(r1), \"=f\"(r2), \"=f\"(r3), \"=f\"(r4), \"=f\"(r5), \"=f\"(r6),"
         " \"=f\"(r7) : \"l\"(p)); }\n";
    o << "static __device__ __forceinline__ float ls_ld_f16(const void* p, int i) {"
         " ls_u16 h = " << (e.l2_keep ? "ls_ldk_u16" : "__ldg") << "((const ls_u16*)p + i); float f; asm(\"cvt.f32.f16 %0, %1;\" : \"=f\"(f) : \"h\"(h));"
         " return f; }\n";
    o << "struct LsEvalArgs { const float* pts; float* out; float* grad; const void* coef;"
         " long long n; int e0, e1, e2, cstride, cunit; unsigned* status; float* hess; const void* tmap; };\n";
    o << "struct LsAdjArgs { const float* pts; const float* gout; float* dcoef;"
         " long long n; int e0, e1, e2, cstride, cunit; unsigned long long* iacc; const float* iscale; };\n";
    o << "struct LsBinArgs { const float* pts; const float* gout; unsigned* key; int* idx; float4* rec;"
         " long long n; int e0, e1, e2, halo; unsigned nbins; };\n";
    o << "struct LsGatherArgs { const float4* srec; const unsigned* start; float* dcoef;"
         " int e0, e1, e2, cstride, cunit, halo; };\n";
    // bounded wait for the completion of an mbarrier phase: gives up after about
    // a second, sets *status to 1 and returns false (the caller's warp leaves)
    o << "static __device__ __forceinline__ bool ls_mbar_wait(unsigned bar, unsigned parity, unsigned* status) {\n"
         "  for (int it = 0; it < " << e.wait_rounds << "; ++it) {\n"
         "    unsigned ok;\n"
         "    asm volatile(\"{ .reg .pred p; mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, 1000;"
         " selp.u32 %0, 1, 0, p; }\" : \"=r\"(ok) : \"r\"(bar), \"r\"(parity) : \"memory\");\n"
         "    if (ok) return true;\n"
         "  }\n"
         "  if (status) atomicOr(status, 1u);\n"
         "  return false;\n"
         "}\n";
    // wait for an mbarrier phase by one thread (the others wait at a barrier):
    // try_wait suspends the thread for a system-dependent time while the phase
    // is incomplete; bounded, sets *status and returns false when it gives up
    o << "static __device__ __forceinline__ bool ls_mbar_poll(unsigned bar, unsigned parity, unsigned* status) {\n"
         "  for (int it = 0; it < " << 4LL * e.wait_rounds << "; ++it) {\n"
         "    unsigned ok;\n"
         "    asm volatile(\"{ .reg .pred p; mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;"
         " selp.u32 %0, 1, 0, p; }\" : \"=r\"(ok) : \"r\"(bar), \"r\"(parity) : \"memory\");\n"
         "    if (ok) return true;\n"
         "  }\n"
         "  if (status) atomicOr(status, 1u);\n"
         "  return false;\n"
         "}\n";
    // warp-aggregated scatter-add: lanes with the same address sum their values
    // by shuffles (per-lane source lanes, warp-uniform trip count) and the
    // lowest of them issues one atomic; ad < 0 means no site (nothing added)
    o << "static __device__ __forceinline__ void ls_agg_add(float* base, int ad, float v) {\n"
         "  const unsigned am = __activemask();\n"
         "  const unsigned peers = __match_any_sync(am, ad);\n"
         "  const unsigned lane = threadIdx.x & 31u;\n"
         "  const int mx = (int)__reduce_max_sync(am, (unsigned)__popc(peers));\n"
         "  float s = v;\n"
         "  unsigned rest = peers & ~(1u << lane);\n"
         "  for (int k = 1; k < mx; ++k) {\n"
         "    const int src = rest ? __ffs(rest) - 1 : (int)lane;\n"
         "    const float o = __shfl_sync(am, v, src);\n"
         "    if (rest) { s += o; rest &= rest - 1u; }\n"
         "  }\n"
         "  if (ad >= 0 && (peers & ((1u << lane) - 1u)) == 0u) atomicAdd(base + ad, s);\n"
         "}\n";
    o << "#define LS_CSWAP(A, B, PA, PB, NA, NB) { bool sw_ = (A) < (B); float ta_ = sw_ ? (B) : (A);"
         " float tb_ = sw_ ? (A) : (B); int pa_ = sw_ ? (PB) : (PA); int pb_ = sw_ ? (PA) : (PB);"
         " unsigned na_ = sw_ ? (NB) : (NA); unsigned nb_ = sw_ ? (NA) : (NB);"
         " A = ta_; B = tb_; PA = pa_; PB = pb_; NA = na_; NB = nb_; }\n";
}

// ---------------------------------------------------------------------------
// point classification: region of evaluation + fold + sub-region
// Emits, inside a point loop with x0..x{dim-1} loaded:
//   int k0..; float y0..; (fold) float a0..; int p0..; unsigned g0.. (sign of
//   reference axis r); int ri0.. (reference axis landing on Cartesian axis i);
//   unsigned ng0.. (sign of Cartesian axis i); int psi;
// ---------------------------------------------------------------------------
void emit_classify(Emitter &e, const Table &t, const char *kshift = nullptr)
{
    auto &o = e.o;
    const int D = t.dim;
    // the two 3D lattices stored as cosets of 2Z^3 whose nearest site has a
    // closed form: BCC = 2Z^3 u (2Z^3 + (1,1,1)), FCC = D3 (integer points
    // with an even coordinate sum)
    auto has_cosets = [&](std::vector<I3> want) {
        if (D != 3 || t.scale != 2 || t.cosets.size() != want.size()) return false;
        for (const auto &c : t.cosets) {
            auto it = std::find(want.begin(), want.end(), I3{c[0], c[1], c[2]});
            if (it == want.end()) return false;
            want.erase(it);
        }
        return true;
    };
    const bool bcc = t.roe != LS_ROE_PARALLELEPIPED && has_cosets({I3{0, 0, 0}, I3{1, 1, 1}});
    const bool fcc = t.roe != LS_ROE_PARALLELEPIPED &&
                     has_cosets({I3{0, 0, 0}, I3{1, 1, 0}, I3{1, 0, 1}, I3{0, 1, 1}});
    if (t.roe == LS_ROE_PARALLELEPIPED) {
        for (int i = 0; i < D; ++i)
            o << "    const float kf" << i << " = floorf(x" << i << ");\n";
    } else if (bcc) {
        // nearest even site c; the nearest odd site is c + sign(x - c) per axis,
        // and it is nearer iff sum |x - c| > 3/2 (|x - c'|^2 - |x - c|^2 =
        // 3 - 2 sum |x - c|)
        for (int i = 0; i < 3; ++i) {
            o << "    const float ce" << i << " = 2.0f * rintf(x" << i << " * 0.5f);\n";
            o << "    const float de" << i << " = x" << i << " - ce" << i << ";\n";
        }
        o << "    const bool odd_ = fabsf(de0) + fabsf(de1) + fabsf(de2) > 1.5f;\n";
        for (int i = 0; i < 3; ++i)
            o << "    const float kf" << i << " = odd_ ? ce" << i << " + (de" << i << " < 0.0f ? -1.0f : 1.0f) : ce"
              << i << ";\n";
    } else if (fcc) {
        // D3: round every coordinate; if the sum of the rounded coordinates is
        // odd, move the coordinate with the largest rounding error to the other
        // neighbouring integer
        for (int i = 0; i < 3; ++i) {
            o << "    const float rr" << i << " = rintf(x" << i << ");\n";
            o << "    const float ee" << i << " = x" << i << " - rr" << i << ";\n";
        }
        o << "    const bool oddsum_ = ((__float2int_rn(rr0) + __float2int_rn(rr1) + __float2int_rn(rr2)) & 1) != 0;\n";
        o << "    const float ae0_ = fabsf(ee0), ae1_ = fabsf(ee1), ae2_ = fabsf(ee2);\n";
        o << "    const int mx_ = (ae0_ >= ae1_ && ae0_ >= ae2_) ? 0 : (ae1_ >= ae2_ ? 1 : 2);\n";
        for (int i = 0; i < 3; ++i)
            o << "    const float kf" << i << " = (oddsum_ && mx_ == " << i << ") ? rr" << i << " + (ee" << i
              << " < 0.0f ? -1.0f : 1.0f) : rr" << i << ";\n";
    } else {
        for (size_t j = 0; j < t.cosets.size(); ++j) {
            for (int i = 0; i < D; ++i) {
                int l = t.cosets[j][i];
                if (t.scale == 1)
                    o << "    const float c" << j << "_" << i << " = rintf(x" << i << ");\n";
                else
                    o << "    const float c" << j << "_" << i << " = fmaf(" << flit(t.scale) << ", rintf((x"
                      << i << " - " << flit(l) << ") * " << flit(1.0 / t.scale) << "), " << flit(l) << ");\n";
            }
            o << "    const float d" << j << " = ";
            for (int i = 0; i < D; ++i)
                o << (i ? " + " : "") << "(x" << i << " - c" << j << "_" << i << ") * (x" << i << " - c" << j
                  << "_" << i << ")";
            o << ";\n";
        }
        for (int i = 0; i < D; ++i) o << "    float kf" << i << " = c0_" << i << ";\n";
        o << "    float dbest = d0;\n";
        for (size_t j = 1; j < t.cosets.size(); ++j) {
            o << "    { const bool b = d" << j << " < dbest; dbest = b ? d" << j << " : dbest;";
            for (int i = 0; i < D; ++i) o << " kf" << i << " = b ? c" << j << "_" << i << " : kf" << i << ";";
            o << " }\n";
        }
    }
    // kshift: k is taken relative to an integer origin (tile-local sites); y,
    // the fold and the sub-region do not change
    for (int i = 0; i < D; ++i) {
        o << "    const int k" << i << " = (int)kf" << i;
        if (kshift) o << " - " << kshift << i;
        o << ";\n";
        o << "    const float y" << i << " = x" << i << " - kf" << i << ";\n";
    }
    if (t.fold == LS_FOLD_SIGNED_PERM) {
        for (int i = 0; i < D; ++i) {
            o << "    const unsigned ng" << i << " = y" << i << " < 0.0f;\n";
            o << "    float a" << i << " = fabsf(y" << i << "); int p" << i << " = " << i << "; unsigned g" << i
              << " = ng" << i << ";\n";
        }
        if (D == 3) {
            o << "    LS_CSWAP(a0, a1, p0, p1, g0, g1); LS_CSWAP(a1, a2, p1, p2, g1, g2);"
                 " LS_CSWAP(a0, a1, p0, p1, g0, g1);\n";
        } else {
            o << "    LS_CSWAP(a0, a1, p0, p1, g0, g1);\n";
        }
        for (int i = 0; i < D; ++i) {
            o << "    const int ri" << i << " = ";
            for (int r = 0; r < D - 1; ++r) o << "(p" << r << " == " << i << ") ? " << r << " : ";
            o << (D - 1) << ";\n";
        }
    } else {
        for (int i = 0; i < D; ++i)
            o << "    const float a" << i << " = y" << i << ";\n";
    }
    // reference sub-region
    if (t.ref.size() > 1) {
        o << "    unsigned q = 0u;\n";
        for (size_t pi = 0; pi < t.planes.size(); ++pi) {
            o << "    q |= (";
            for (int i = 0; i < D; ++i) o << (i ? " + " : "") << flit(t.planes[pi][i]) << " * a" << i;
            o << " - " << flit(t.planes[pi][3]) << " >= 0.0f) ? " << (1u << pi) << "u : 0u;\n";
        }
        unsigned long long packed = 0;
        for (int qq = 0; qq < t.bsp_mod; ++qq) {
            unsigned v = t.sigma[qq] < 0 ? 0u : (unsigned)t.sigma[qq];
            packed |= (unsigned long long)(v & 0xF) << (4 * qq);
        }
        o << "    const int psi = (int)((" << packed << "ull >> (4u * (q % " << t.bsp_mod << "u))) & 15ull);\n";
    } else {
        o << "    const int psi = 0;\n";
    }
}

// coset id LUT packed by parity pattern (scale 2) -> coset index
unsigned long long coset_lut(const Table &t)
{
    unsigned long long lut = ~0ull;
    for (size_t j = 0; j < t.cosets.size(); ++j) {
        int par = 0;
        for (int i = 0; i < t.dim; ++i) par |= (t.cosets[j][i] & 1) << i;
        lut &= ~(0xFull << (4 * par));
        lut |= (unsigned long long)j << (4 * par);
    }
    return lut;
}

// ---------------------------------------------------------------------------
// Copy choice for the shifted bricked copies.
//
// A point's stencil is a fixed set of sites around its region-of-evaluation
// site k, placed by the point's signed permutation; how many 32-byte sectors
// it touches depends on where the brick boundaries cut it.  The four copies
// shift the brick grid by (s_0, s_1) in {0,1}^2 grid indices.  The choice is
// made per Cartesian axis i in {0, 1} from what fixes the stencil's position
// along that axis: the reference sub-region psi, the reference axis r landing
// on axis i, its sign, and k_i mod 4; bit key(psi, r, neg, k_i mod 4) of a
// 64-bit mask per axis holds s_i.  The masks minimise the sectors summed over
// all classes (sub-region, transform, k mod 4 on each axis over the lattice's
// sites), alternating between the two axes from s = 0.
// ---------------------------------------------------------------------------
int shift_key(int psi, int r, int neg, int kmod4) { return ((psi * 3 + r) * 2 + neg) * 4 + kmod4; }

struct ShiftRule {
    unsigned long long mask[3] = {0, 0, 0};
    double base = 0.0, best = 0.0;        // mean sectors per class: copy 0 only, with the rule
};

// nax = 2: copies shifted on x and y (4); nax = 3: also on z (8).
ShiftRule shift_rule(const Table &t, const std::vector<std::vector<I3>> &region_sites, int elem_bytes, int nax)
{
    ShiftRule rule;
    const bool fold = t.fold == LS_FOLD_SIGNED_PERM;
    const int a = t.scale;
    const int C = (int)t.cosets.size();
    const int per_sector = 32 / elem_bytes;
    const int ncopy = 1 << nax;
    struct Cls { int key[3]; std::vector<int> cnt; };
    std::vector<Cls> cls;
    int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    const int np = fold ? 6 : 1, ns = fold ? 8 : 1;
    for (size_t psi = 0; psi < region_sites.size(); ++psi)
        for (int pi = 0; pi < np; ++pi)
            for (int sg = 0; sg < ns; ++sg)
                for (int km = 0; km < 64; ++km) {
                    const int kq[3] = {km & 3, (km >> 2) & 3, (km >> 4) & 3};
                    if (a == 2) {        // k must be a lattice site: its parity pattern is a coset's
                        int par = (kq[0] & 1) | ((kq[1] & 1) << 1) | ((kq[2] & 1) << 2), hit = 0;
                        for (const auto &l : t.cosets)
                            hit |= ((l[0] & 1) | ((l[1] & 1) << 1) | ((l[2] & 1) << 2)) == par;
                        if (!hit) continue;
                    }
                    const int *p = perms[pi];           // reference axis r lands on Cartesian axis p[r]
                    const int g[3] = {sg & 1, (sg >> 1) & 1, (sg >> 2) & 1};   // sign bit of reference axis r
                    // more than two sub-regions do not fit the 64-bit key: the rule then ignores psi
                    const int pk = region_sites.size() <= 2 ? (int)psi : 0;
                    Cls c;
                    for (int r = 0; r < 3; ++r) c.key[p[r]] = shift_key(pk, r, g[r], kq[p[r]]);
                    c.cnt.assign(ncopy, 0);
                    for (int cp = 0; cp < ncopy; ++cp) {
                        std::set<long long> sec;
                        for (const auto &sref : region_sites[psi]) {
                            int n[3];
                            for (int i = 0; i < 3; ++i) n[i] = 64 + kq[i];
                            for (int r = 0; r < 3; ++r) n[p[r]] += g[r] ? -sref[r] : sref[r];
                            int j = 0, q[3];
                            if (a == 2) {
                                const int par = (n[0] & 1) | ((n[1] & 1) << 1) | ((n[2] & 1) << 2);
                                for (size_t cc = 0; cc < t.cosets.size(); ++cc)
                                    if (((t.cosets[cc][0] & 1) | ((t.cosets[cc][1] & 1) << 1) |
                                         ((t.cosets[cc][2] & 1) << 2)) == par)
                                        j = (int)cc;
                                for (int i = 0; i < 3; ++i) q[i] = n[i] >> 1;
                            } else {
                                for (int i = 0; i < 3; ++i) q[i] = n[i];
                            }
                            for (int i = 0; i < nax; ++i) q[i] += (cp >> i) & 1;
                            const long long bk = (q[0] >> 1) + 1000LL * ((q[1] >> 1) + 1000LL * (q[2] >> 1));
                            const int w = (q[0] & 1) + 2 * (q[1] & 1) + 4 * (q[2] & 1);
                            sec.insert(((bk * 8 + w) * C + j) / per_sector);
                        }
                        c.cnt[cp] = (int)sec.size();
                    }
                    cls.push_back(c);
                }
    if (cls.empty()) return rule;
    std::vector<std::vector<int>> rr(3, std::vector<int>(64, 0));
    auto copy_of = [&](const Cls &c, int axis, int bit) {
        int cp = 0;
        for (int i = 0; i < nax; ++i) cp |= (i == axis ? bit : rr[i][c.key[i]]) << i;
        return cp;
    };
    for (int it = 0; it < 4; ++it)
        for (int axis = 0; axis < nax; ++axis) {
            std::vector<long long> tot0(64, 0), tot1(64, 0);
            for (const auto &c : cls) {
                tot0[c.key[axis]] += c.cnt[copy_of(c, axis, 0)];
                tot1[c.key[axis]] += c.cnt[copy_of(c, axis, 1)];
            }
            for (int k = 0; k < 64; ++k) rr[axis][k] = tot1[k] < tot0[k] ? 1 : 0;
        }
    double base = 0, best = 0;
    for (const auto &c : cls) {
        base += c.cnt[0];
        best += c.cnt[copy_of(c, 0, rr[0][c.key[0]])];
    }
    for (int i = 0; i < nax; ++i)
        for (int k = 0; k < 64; ++k) rule.mask[i] |= (unsigned long long)rr[i][k] << k;
    rule.base = base / (double)cls.size();
    rule.best = best / (double)cls.size();
    return rule;
}

// The site lists the gathers of each reference sub-region read (the product
// stencil of a tensor-product spline), for the copy-choice rule.
void setup_brick_shift(Emitter &e, const Table &t, int brick, ls_dtype dt)
{
    e.brick_shift = brick == 2 || brick == 3;
    e.shift_axes = brick == 3 ? 3 : 2;
    if (!e.brick_shift) return;
    std::vector<std::vector<I3>> rs;
    if (!t.sep.empty()) {
        std::vector<I3> sites;
        for (int s2 : t.sep[2].sites)
            for (int s1 : t.sep[1].sites)
                for (int s0 : t.sep[0].sites) sites.push_back({s0, s1, s2});
        rs.push_back(sites);
    } else {
        for (const auto &r : t.ref) rs.push_back(r.sites);
    }
    const ShiftRule rule = shift_rule(t, rs, dt == LS_F32 ? 4 : 2, e.shift_axes);
    for (int i = 0; i < 3; ++i) e.shift_mask[i] = rule.mask[i];
}

// ---------------------------------------------------------------------------
// addressing + gathers: emits float cN = coefficient of union site N.
// Fast path with unchecked addresses when the whole stencil is inside;
// checked path otherwise.
// ---------------------------------------------------------------------------
// load: emit float cN = coefficient; declare_addr: emit int adN = address (-1 if
// the site is outside the arrays).  At least one of the two is set.
void emit_gathers(Emitter &e, const Table &t, const std::vector<I3> &sites, int reach,
                  const char *coef_expr, bool declare_addr, bool load = true, int group = 0, int depth = 0)
{
    auto &o = e.o;
    const int D = t.dim;
    const bool fold = t.fold == LS_FOLD_SIGNED_PERM;
    const int a = t.scale;
    // Vector gathers: on the eight shifted copies a Cartesian stencil that is a
    // box (contiguous extent per axis) starts on a brick boundary in the copy
    // chosen by the parity of its first site, so it lies in a box of whole
    // 2 x 2 x 2 bricks, each 32 contiguous bytes: one 32-byte load per brick.
    // An odd extent n reads (n + 1) / 2 bricks, the last one's far half unused
    // (inside the copy: its padding of two planes per axis holds it).
    int vlo[3] = {0, 0, 0}, vn[3] = {1, 1, 1};
    bool vec = e.brick_shift && e.shift_axes == 3 && D == 3 && a == 1 && t.cosets.size() == 1 && load &&
               !declare_addr && group == 0 && e.ld == "ls_ld_f32" && !fold && !sites.empty();
    if (vec) {
        for (int i = 0; i < 3; ++i) {
            std::set<int> vals;
            for (const auto &sv : sites) vals.insert(sv[i]);
            vlo[i] = *vals.begin();
            vn[i] = (int)vals.size();
            vec = vec && *vals.rbegin() - vlo[i] + 1 == vn[i];
        }
        vec = vec && (size_t)(vn[0] * vn[1] * vn[2]) == sites.size();
    }
    o << "    const int ex0 = E0, ex1 = E1" << (D == 3 ? ", ex2 = E2" : "") << ";\n";
    o << "    bool inside = true;\n";
    for (int i = 0; i < D; ++i)
        o << "    inside = inside && (k" << i << " - " << reach << " >= 0) && (k" << i << " + " << reach
          << " <= " << a << " * ex" << i << " - 1);\n";
    if (load)
        for (size_t j = 0; j < sites.size(); ++j) o << "    float c" << j << ";\n";
    if (declare_addr)
        for (size_t j = 0; j < sites.size(); ++j) o << "    int ad" << j << ";\n";
    // Address of (coset j, per-coset index q).  Linear layouts (coset-major,
    // interleaved): j * CS + CU * (q0 + ex0 (q1 + ex1 q2)).  Bricked layout
    // (2 x 2 x 2 indices per brick, cosets interleaved inside, e.brick):
    // j + sum_i [BA_i q_i + BB_i (q_i >> 1)], which is BH_i (q_i >> 1) +
    // BA_i (q_i & 1) per axis.
    if (e.brick) {
        o << "    const int BA0 = CU, BA1 = 2 * CU, BA2 = 4 * CU;\n";
        if (e.brick_shift) {
            // the shifted copies: bricks over the padded extents, copy (sx, sy[, sz])
            // chosen per point (shift_rule), Q = CS elements per copy
            o << "    const int BH0 = 8 * CU, BH1 = BH0 * ((ex0 + 2) >> 1), BH2 = BH1 * ((ex1 + 2) >> 1);\n";
            auto key = [&](int i) {
                const std::string r = fold ? "ri" + std::to_string(i) : std::to_string(i);
                const std::string ng = fold ? "(int)ng" + std::to_string(i) : "0";
                const std::string ps = t.ref.size() <= 2 ? "psi" : "0";
                return "((" + ps + " * 3 + " + r + ") * 2 + " + ng + ") * 4 + (k" + std::to_string(i) + " & 3)";
            };
            const char *sn[3] = {"sx", "sy", "sz"};
            for (int i = 0; i < e.shift_axes; ++i) {
                if (vec)   // the copy in which the stencil starts on a brick boundary on every axis
                    o << "    const int " << sn[i] << " = (k" << i << " + (" << vlo[i] << ")) & 1;\n";
                else
                    o << "    const int " << sn[i] << " = (int)((" << e.shift_mask[i] << "ull >> (" << key(i)
                      << ")) & 1ull);\n";
            }
            if (e.shift_axes == 3) o << "    const int cbase = (sx + 2 * sy + 4 * sz) * CS;\n";
            else o << "    const int cbase = (sx + 2 * sy) * CS;\n";
        } else {
            o << "    const int BH0 = " << (D == 3 ? 8 : 4) << " * CU, BH1 = BH0 * (ex0 >> 1), BH2 = BH1 * (ex1 >> 1);\n";
        }
        o << "    const int BB0 = BH0 - 2 * BA0, BB1 = BH1 - 2 * BA1, BB2 = BH2 - 2 * BA2;\n";
        o << "    (void)BA2; (void)BB2;\n";
    }
    o << "    if (inside) {\n";
    if (vec) {
        o << "      const float* vb_ = (const float*)" << coef_expr << " + cbase + ((k0 + (" << vlo[0]
          << ") + sx) >> 1) * BH0 + ((k1 + (" << vlo[1] << ") + sy) >> 1) * BH1 + ((k2 + (" << vlo[2]
          << ") + sz) >> 1) * BH2;\n";
        for (int b2 = 0; b2 < (vn[2] + 1) / 2; ++b2)
            for (int b1 = 0; b1 < (vn[1] + 1) / 2; ++b1)
                for (int b0 = 0; b0 < (vn[0] + 1) / 2; ++b0) {
                    const std::string nm = "vq" + std::to_string(b0) + std::to_string(b1) + std::to_string(b2);
                    const std::string off = std::to_string(b0) + " * BH0 + " + std::to_string(b1) + " * BH1 + " +
                                            std::to_string(b2) + " * BH2";
                    o << "      float " << nm << "_0";
                    for (int w = 1; w < 8; ++w) o << ", " << nm << "_" << w;
                    o << ";\n      ls_ld8(vb_ + " << off;
                    for (int w = 0; w < 8; ++w) o << ", " << nm << "_" << w;
                    o << ");\n";
                }
        for (size_t j = 0; j < sites.size(); ++j) {
            const int o0 = sites[j][0] - vlo[0], o1 = sites[j][1] - vlo[1], o2 = sites[j][2] - vlo[2];
            const int w = (o0 & 1) + 2 * (o1 & 1) + 4 * (o2 & 1);
            o << "      c" << j << " = vq" << (o0 >> 1) << (o1 >> 1) << (o2 >> 1) << "_" << w << ";\n";
        }
    } else {
    // strides of the reference axes (the linear part)
    const char *st_lin[3] = {"CU", "(CU * ex0)", "(CU * ex0 * ex1)"};
    const char *st_brk[3] = {"BA0", "BA1", "BA2"};
    const char *const *st = e.brick ? st_brk : st_lin;
    for (int r = 0; r < D; ++r) {
        if (fold) {
            o << "      int rs" << r << " = ";
            for (int i = 0; i < D - 1; ++i) o << "(p" << r << " == " << i << ") ? " << st[i] << " : ";
            o << st[D - 1] << ";\n";
            o << "      rs" << r << " = g" << r << " ? -rs" << r << " : rs" << r << ";\n";
        } else {
            o << "      const int rs" << r << " = " << st[r] << ";\n";
        }
    }
    if (e.brick) {
        // per reference axis: the Cartesian axis' brick shift and coefficient, the sign
        const char *bb[3] = {"BB0", "BB1", "BB2"};
        for (int r = 0; r < D; ++r) {
            if (fold) {
                o << "      const int bsh" << r << " = 1;\n";
                o << "      const int bbt" << r << " = ";
                for (int i = 0; i < D - 1; ++i) o << "(p" << r << " == " << i << ") ? " << bb[i] << " : ";
                o << bb[D - 1] << ";\n";
                o << "      const int bsg" << r << " = g" << r << " ? -1 : 1;\n";
            } else {
                o << "      const int bsh" << r << " = 1, bbt" << r << " = " << bb[r]
                  << ", bsg" << r << " = 1;\n";
            }
        }
    }
    // parity classes
    std::map<int, std::string> base_of_class;
    auto parity_class = [&](const I3 &s) {
        int m = 0;
        if (a == 2)
            for (int r = 0; r < D; ++r) m |= (s[r] & 1) << r;
        return m;
    };
    auto hoff = [&](const I3 &s, int r) { return (a == 2) ? floordiv2(s[r]) : s[r]; };
    // the per-class grid index of the class' h = 0 site on each Cartesian axis
    // (Q<m>_<i>) and its coset id; the base address of the class
    auto emit_brick_class = [&](int m, const std::string &qexpr0, const std::string &qexpr1,
                                const std::string &qexpr2, const std::string &cidexpr) {
        const std::string qx[3] = {qexpr0, qexpr1, qexpr2};
        for (int i = 0; i < D; ++i) o << "      const int Q" << m << "_" << i << " = " << qx[i] << ";\n";
        // grid index on reference axis r: Q<m>_{p_r}
        for (int r = 0; r < D; ++r) {
            o << "      const int QR" << m << "_" << r << " = ";
            if (fold) {
                for (int i = 0; i < D - 1; ++i) o << "(p" << r << " == " << i << ") ? Q" << m << "_" << i << " : ";
                o << "Q" << m << "_" << (D - 1) << ";\n";
            } else {
                o << "Q" << m << "_" << r << ";\n";
            }
        }
        std::string nm = "base" + std::to_string(m);
        o << "      const int " << nm << " = " << cidexpr;
        for (int i = 0; i < D; ++i) o << " + BA" << i << " * Q" << m << "_" << i;
        o << ";\n";
        // nonlinear terms of every offset h used by this class on axis r
        std::set<std::pair<int, int>> used;
        for (const auto &sv : sites)
            if (parity_class(sv) == m)
                for (int r = 0; r < D; ++r) used.insert({r, hoff(sv, r)});
        for (const auto &rh : used) {
            const int r = rh.first, h = rh.second;
            o << "      const int nl" << m << "_" << r << "_" << (h < 0 ? "m" : "") << std::abs(h) << " = bbt" << r
              << " * ((QR" << m << "_" << r << " + bsg" << r << " * (" << h << ")) >> bsh" << r << ");\n";
        }
        base_of_class[m] = nm;
    };
    if (a == 1) {
        if (e.brick_shift) {
            emit_brick_class(0, "(k0 + sx)", "(k1 + sy)", e.shift_axes == 3 ? "(k2 + sz)" : "k2", "cbase");
        } else if (e.brick) {
            emit_brick_class(0, "k0", D >= 2 ? "k1" : "0", D == 3 ? "k2" : "0", "0");
        } else {
            o << "      const int base0 = CU * (";
            o << "k0" << (D >= 2 ? " + ex0 * (k1" : "") << (D == 3 ? " + ex1 * k2" : "") << (D >= 2 ? ")" : "")
              << ");\n";
            base_of_class[0] = "base0";
        }
    } else {
        const unsigned long long lut = coset_lut(t);
        for (int i = 0; i < D; ++i)
            if (e.brick_shift && i < e.shift_axes)
                o << "      const int qh" << i << " = (k" << i << " >> 1) + " << (i == 0 ? "sx" : i == 1 ? "sy" : "sz")
                  << ", cb" << i << " = k" << i << " & 1;\n";
            else
                o << "      const int qh" << i << " = k" << i << " >> 1, cb" << i << " = k" << i << " & 1;\n";
        std::set<int> classes;
        for (const auto &s : sites) classes.insert(parity_class(s));
        for (int m : classes) {
            std::string nm = "base" + std::to_string(m);
            for (int i = 0; i < D; ++i) {
                // component of R^T e on Cartesian axis i: e[ri_i], negated if axis i is negative
                if (fold)
                    o << "      const int ce" << m << "_" << i << " = "
                      << (m == 0 ? std::string("0") : m == (1 << D) - 1 ? std::string("1")
                                                       : "(" + std::to_string(m) + " >> ri" + std::to_string(i) + ") & 1")
                      << ";\n";
                else
                    o << "      const int ce" << m << "_" << i << " = " << ((m >> i) & 1) << ";\n";
                o << "      const int v" << m << "_" << i << " = cb" << i << " + "
                  << (fold ? ("(ng" + std::to_string(i) + " ? -ce" + std::to_string(m) + "_" + std::to_string(i) +
                              " : ce" + std::to_string(m) + "_" + std::to_string(i) + ")")
                           : ("ce" + std::to_string(m) + "_" + std::to_string(i)))
                  << ";\n";
            }
            o << "      const int par" << m << " = (v" << m << "_0 & 1)";
            for (int i = 1; i < D; ++i) o << " | ((v" << m << "_" << i << " & 1) << " << i << ")";
            o << ";\n";
            o << "      const int cid" << m << " = (int)((" << (lut & 0xFFFFFFFFull) << "u >> (4 * par" << m << ")) & 15u);\n";
            auto q = [&](int i) {
                return i < D ? "qh" + std::to_string(i) + " + (v" + std::to_string(m) + "_" + std::to_string(i) + " >> 1)"
                             : std::string("0");
            };
            if (e.brick) {
                emit_brick_class(m, q(0), q(1), q(2), (e.brick_shift ? "cbase + cid" : "cid") + std::to_string(m));
            } else {
                o << "      const int " << nm << " = cid" << m << " * CS + CU * ((" << q(0) << ")";
                if (D >= 2) o << " + ex0 * ((" << q(1) << ")";
                if (D == 3) o << " + ex1 * (" << q(2) << ")";
                if (D >= 2) o << ")";
                o << ");\n";
                base_of_class[m] = nm;
            }
        }
    }
    const bool pipelined = load && !declare_addr && group > 0 && depth > 0 && (int)sites.size() > group * depth;
    for (size_t j = 0; j < sites.size(); ++j) {
        const I3 &s = sites[j];
        const int m = parity_class(s);
        std::string addr = base_of_class[m];
        if (pipelined && (int)j % group == 0 && (int)j / group >= depth) {
            // Algorithm 2: group g is fetched only once group g - depth has arrived.
            // tk is 0 for every value (NaN and +-inf convert to 0) but is computed
            // from the loaded value, so the loads below cannot issue before it.
            const int g = (int)j / group;
            const int last = (g - depth + 1) * group - 1;
            o << "      const int tk" << g << " = __float2int_rz(c" << last << " * 0.0f);\n";
        }
        if (pipelined && (int)j / group >= depth) addr += " + tk" + std::to_string((int)j / group);
        for (int r = 0; r < D; ++r) {
            int h = hoff(s, r);
            if (e.brick)
                addr += " + nl" + std::to_string(m) + "_" + std::to_string(r) + "_" + (h < 0 ? "m" : "") +
                        std::to_string(std::abs(h));
            if (h == 0) continue;
            if (h == 1) addr += " + rs" + std::to_string(r);
            else if (h == -1) addr += " - rs" + std::to_string(r);
            else addr += " + (" + std::to_string(h) + ") * rs" + std::to_string(r);
        }
        if (declare_addr) {
            o << "      ad" << j << " = " << addr << ";\n";
            if (load) o << "      c" << j << " = " << e.ld << "(" << coef_expr << ", ad" << j << ");\n";
        } else {
            o << "      c" << j << " = " << e.ld << "(" << coef_expr << ", " << addr << ");\n";
        }
    }
    }
    o << "    } else {\n";
    for (size_t j = 0; j < sites.size(); ++j) {
        const I3 &s = sites[j];
        o << "      {\n";
        for (int i = 0; i < D; ++i) {
            if (fold) {
                o << "        const int m" << i << " = ";
                for (int r = 0; r < D - 1; ++r) o << "(ri" << i << " == " << r << ") ? " << s[r] << " : ";
                o << s[D - 1] << ";\n";
                o << "        const int n" << i << " = k" << i << " + (ng" << i << " ? -m" << i << " : m" << i
                  << ");\n";
            } else {
                o << "        const int n" << i << " = k" << i << " + " << s[i] << ";\n";
            }
        }
        o << "        const bool ok = ";
        for (int i = 0; i < D; ++i)
            o << (i ? " && " : "") << "((unsigned)n" << i << " < (unsigned)(" << a << " * ex" << i << "))";
        o << ";\n";
        if (a == 2) {
            const unsigned long long lut = coset_lut(t);
            o << "        const int par = (n0 & 1)";
            for (int i = 1; i < D; ++i) o << " | ((n" << i << " & 1) << " << i << ")";
            o << ";\n        const int cid = (int)((" << (lut & 0xFFFFFFFFull) << "u >> (4 * par)) & 15u);\n";
            if (e.brick) {
                o << "        const int adr = " << (e.brick_shift ? "cbase + cid" : "cid");
                for (int i = 0; i < D; ++i) {
                    if (e.brick_shift && i < e.shift_axes) {
                        const std::string g = "((n" + std::to_string(i) + " >> 1) + " +
                                              (i == 0 ? "sx)" : i == 1 ? "sy)" : "sz)");
                        o << " + BA" << i << " * " << g << " + BB" << i << " * (" << g << " >> 1)";
                    } else {
                        o << " + BA" << i << " * (n" << i << " >> 1) + BB" << i << " * ((n" << i << " >> 1) >> 1)";
                    }
                }
                o << ";\n";
            } else {
                o << "        const int adr = cid * CS + CU * ((n0 >> 1)";
                if (D >= 2) o << " + ex0 * ((n1 >> 1)";
                if (D == 3) o << " + ex1 * (n2 >> 1)";
                if (D >= 2) o << ")";
                o << ");\n";
            }
        } else {
            if (e.brick) {
                o << "        const int adr = " << (e.brick_shift ? "cbase" : "0");
                for (int i = 0; i < D; ++i) {
                    if (e.brick_shift && i < e.shift_axes) {
                        const std::string g = "(n" + std::to_string(i) + (i == 0 ? " + sx)" : i == 1 ? " + sy)" : " + sz)");
                        o << " + BA" << i << " * " << g << " + BB" << i << " * (" << g << " >> 1)";
                    } else {
                        o << " + BA" << i << " * n" << i << " + BB" << i << " * (n" << i << " >> 1)";
                    }
                }
                o << ";\n";
            } else {
                o << "        const int adr = CU * (n0";
                if (D >= 2) o << " + ex0 * (n1";
                if (D == 3) o << " + ex1 * n2";
                if (D >= 2) o << ")";
                o << ");\n";
            }
        }
        if (declare_addr) o << "        ad" << j << " = ok ? adr : -1;\n";
        if (load) o << "        c" << j << " = ok ? " << e.ld << "(" << coef_expr << ", adr) : 0.0f;\n";
        o << "      }\n";
    }
    o << "    }\n";
}

// ---------------------------------------------------------------------------
// polynomial evaluation in coefficient form + multivariate Horner
// ---------------------------------------------------------------------------
struct PolyEmit {
    Emitter &e;
    int D;
    std::string pre;                           // name prefix for this region
    std::string uvar[3];                       // names of the local coordinates
    std::map<I3, std::vector<std::pair<int, double>>> terms;   // monomial -> (union site, coef)
    std::map<I3, std::string> aname;           // emitted A_a

    // A_a = sum_j M[j][a] c_j
    std::string A(const I3 &m)
    {
        auto it = aname.find(m);
        if (it != aname.end()) return it->second;
        auto t = terms.find(m);
        if (t == terms.end() || t->second.empty()) return aname[m] = "";
        std::string nm = pre + "A" + std::to_string(m[0]) + "_" + std::to_string(m[1]) + "_" + std::to_string(m[2]);
        std::string acc;
        for (auto &pr : t->second) {
            if (acc.empty()) {
                acc = flit(pr.second) + " * c" + std::to_string(pr.first);
                e.fma++;
            } else {
                acc = "fmaf(" + flit(pr.second) + ", c" + std::to_string(pr.first) + ", " + acc + ")";
                e.fma++;
            }
        }
        e.o << "    const float " << nm << " = " << acc << ";\n";
        return aname[m] = nm;
    }

    // Horner over variables v..D-1 with fixed exponents for earlier variables.
    // coeff(m) gives the coefficient expression name of monomial m ("" if 0).
    std::string horner(int v, I3 prefix, const std::function<std::string(const I3 &)> &coeff,
                       const std::set<I3> &support)
    {
        if (v >= D || v >= 3) return coeff(prefix);
        int emax = -1;
        for (const auto &m : support) {
            bool match = true;
            for (int i = 0; i < v; ++i)
                if (m[i] != prefix[i]) match = false;
            if (match) emax = std::max(emax, m[v]);
        }
        if (emax < 0) return "";
        std::string acc;
        for (int ex = emax; ex >= 0; --ex) {
            I3 p = prefix;
            p[v] = ex;
            std::string t = horner(v + 1, p, coeff, support);
            if (acc.empty()) {
                acc = t;
                if (!acc.empty() && ex > 0) {
                    // acc will be multiplied next iteration
                }
                continue;
            }
            std::string nm = e.fresh("h");
            if (t.empty()) {
                e.o << "    const float " << nm << " = " << acc << " * " << uvar[v] << ";\n";
            } else {
                e.o << "    const float " << nm << " = fmaf(" << acc << ", " << uvar[v] << ", " << t << ");\n";
            }
            e.fma++;
            acc = nm;
        }
        // leading zeros: if acc became non-empty only at a lower exponent it is already correct
        return acc;
    }
};

// Horner needs care when leading coefficients vanish; rebuild with explicit
// powers handled by multiplying through.  The implementation above starts the
// accumulator at the highest exponent that has a nonzero sub-polynomial: when
// acc is empty at exponent ex, the sub-polynomial of that exponent is zero and
// skipping it is exact because no lower-exponent term has been folded yet.

std::set<I3> monomial_support(const RefRegion &r, const std::vector<int> &umap,
                              std::map<I3, std::vector<std::pair<int, double>>> &terms)
{
    std::set<I3> sup;
    const size_t nm = r.mono.size();
    for (size_t j = 0; j < r.sites.size(); ++j)
        for (size_t a = 0; a < nm; ++a) {
            double c = r.coef[j * nm + a];
            if (c == 0.0) continue;
            terms[r.mono[a]].push_back({umap[j], c});
            sup.insert(r.mono[a]);
        }
    return sup;
}

// ---------------------------------------------------------------------------
// Factored coefficient transform.
//
// The coefficient form needs A = M^T c (A_a = sum_j M[j][a] c_j), one
// multiply-add per nonzero of M.  The columns of M are far from independent:
// the box spline's symmetries (w_j(sigma u) = w_pi(j)(u) for signed
// permutations sigma that preserve the polynomial piece, Sec. 3) make many
// pairs of rows equal or opposite on many monomials.  A butterfly on two
// variables v, w (p = v + w, q = v - w) turns their rows r_v, r_w into
// (r_v + r_w) / 2 and (r_v - r_w) / 2, which are zero wherever r_w = +-r_v.
// Applied greedily (the pair with the largest saving each time, also to the
// outputs of earlier butterflies) this gives A = M'^T (B c), with B a few
// dozen additions and M' much sparser: the same A_a in fewer operations
// (BCC quintic: 377 instead of 1016).  Every intermediate is a sum or
// difference of at most 2^depth coefficients with rows scaled by 2^-depth, so
// the rounding error stays that of the direct sums.
// ---------------------------------------------------------------------------
struct FactoredTransform {
    struct Op { int v, w, p, q; };            // p = v + w, q = v - w (-1: not formed)
    std::vector<std::vector<double>> rows;    // per variable: coefficients over the monomials
    std::vector<Op> ops;
    std::vector<int> live;                    // variables the final dot products read
    int cost = 0;                             // FP32 operations: additions + nonzeros of M'
};

FactoredTransform factor_transform(const RefRegion &r)
{
    FactoredTransform f;
    const size_t nj = r.sites.size(), na = r.mono.size();
    double big = 0.0;
    for (double c : r.coef) big = std::max(big, std::fabs(c));
    const double tiny = 1e-12 * big;
    auto nnz = [&](const std::vector<double> &v) {
        int n = 0;
        for (double x : v) n += x != 0.0;
        return n;
    };
    for (size_t j = 0; j < nj; ++j) {
        f.rows.emplace_back(r.coef.begin() + (long)(j * na), r.coef.begin() + (long)((j + 1) * na));
        if (nnz(f.rows.back())) f.live.push_back((int)j);
    }
    std::vector<double> p(na), q(na), bp(na), bq(na);
    for (;;) {
        int best = 0, bi = -1, bk = -1;
        for (size_t i = 0; i < f.live.size(); ++i)
            for (size_t k = i + 1; k < f.live.size(); ++k) {
                const auto &rv = f.rows[(size_t)f.live[i]], &rw = f.rows[(size_t)f.live[k]];
                int before = 0, np = 0, nq = 0;
                for (size_t a = 0; a < na; ++a) {
                    before += (rv[a] != 0.0) + (rw[a] != 0.0);
                    np += std::fabs(rv[a] + rw[a]) > tiny;
                    nq += std::fabs(rv[a] - rw[a]) > tiny;
                }
                const int gain = before - np - nq - (np > 0) - (nq > 0);
                if (gain > best) best = gain, bi = (int)i, bk = (int)k;
            }
        if (best <= 0) break;
        const int v = f.live[(size_t)bi], w = f.live[(size_t)bk];
        for (size_t a = 0; a < na; ++a) {
            const double x = f.rows[(size_t)v][a], y = f.rows[(size_t)w][a];
            bp[a] = std::fabs(x + y) > tiny ? 0.5 * (x + y) : 0.0;
            bq[a] = std::fabs(x - y) > tiny ? 0.5 * (x - y) : 0.0;
        }
        FactoredTransform::Op op{v, w, -1, -1};
        f.live.erase(f.live.begin() + bk);
        f.live.erase(f.live.begin() + bi);
        if (nnz(bp)) op.p = (int)f.rows.size(), f.rows.push_back(bp), f.live.push_back(op.p), f.cost++;
        if (nnz(bq)) op.q = (int)f.rows.size(), f.rows.push_back(bq), f.live.push_back(op.q), f.cost++;
        f.ops.push_back(op);
    }
    for (int v : f.live) f.cost += nnz(f.rows[(size_t)v]);
    return f;
}

// Emits the butterflies and every nonzero A_a of the region; fills pe.aname
// (the names the Horner forms read).
void emit_factored_transform(Emitter &e, const RefRegion &r, const std::vector<int> &umap,
                             const FactoredTransform &f, PolyEmit &pe)
{
    auto &o = e.o;
    const size_t nj = r.sites.size(), na = r.mono.size();
    auto vname = [&](int v) {
        return (size_t)v < nj ? "c" + std::to_string(umap[(size_t)v]) : pe.pre + "t" + std::to_string(v);
    };
    for (const auto &op : f.ops) {
        if (op.p >= 0) o << "    const float " << vname(op.p) << " = " << vname(op.v) << " + " << vname(op.w) << ";\n";
        if (op.q >= 0) o << "    const float " << vname(op.q) << " = " << vname(op.v) << " - " << vname(op.w) << ";\n";
        e.fma += (op.p >= 0) + (op.q >= 0);
    }
    auto mono_name = [&](size_t a) {
        const I3 &m = r.mono[a];
        return pe.pre + "A" + std::to_string(m[0]) + "_" + std::to_string(m[1]) + "_" + std::to_string(m[2]);
    };
    std::vector<int> partner(na, -1);
    if (e.fma2) {
        // Paired FMA (Blackwell's fma.rn.f32x2): two monomials whose sums read
        // many of the same variables are formed together, one instruction per
        // variable either reads, with the pair of constants from a __constant__
        // table and the variable duplicated into both halves once.  A variable
        // only one of the two reads adds 0 to the other (exact).  Greedy: each
        // monomial in turn takes the free one sharing the most variables, if it
        // shares 2+.  Measured slower than the scalar sums on B300 (a variant).
        std::vector<std::vector<char>> in(na, std::vector<char>(f.rows.size(), 0));
        std::vector<int> cnt(na, 0);
        for (size_t a = 0; a < na; ++a)
            for (int v : f.live)
                if (f.rows[(size_t)v][a] != 0.0) in[a][(size_t)v] = 1, cnt[a]++;
        std::vector<size_t> order(na);
        for (size_t a = 0; a < na; ++a) order[a] = a;
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cnt[x] > cnt[y]; });
        for (size_t a : order) {
            if (partner[a] >= 0 || cnt[a] == 0) continue;
            int best = -1, bshare = 1;
            for (size_t b : order) {
                if (b == a || partner[b] >= 0 || cnt[b] == 0) continue;
                int share = 0;
                for (int v : f.live) share += in[a][(size_t)v] && in[b][(size_t)v];
                if (share > bshare) bshare = share, best = (int)b;
            }
            if (best >= 0) partner[a] = best, partner[(size_t)best] = (int)a;
        }
        std::vector<std::pair<float, float>> kv;
        std::ostringstream body;
        std::set<int> dup;
        std::vector<std::pair<size_t, size_t>> pairs;
        for (size_t a : order)
            if (partner[a] >= 0 && (size_t)partner[a] > a) pairs.push_back({a, (size_t)partner[a]});
        for (const auto &pr : pairs) {
            std::string acc;
            for (int v : f.live) {
                const double ca = f.rows[(size_t)v][pr.first], cb = f.rows[(size_t)v][pr.second];
                if (ca == 0.0 && cb == 0.0) continue;
                if (!dup.count(v)) {
                    body << "    const float2 " << pe.pre << "uu" << v << " = make_float2(" << vname(v) << ", "
                         << vname(v) << ");\n";
                    dup.insert(v);
                }
                const std::string k = "@K[" + std::to_string(kv.size()) + "]";
                kv.push_back({(float)ca, (float)cb});
                const std::string uu = pe.pre + "uu" + std::to_string(v);
                acc = acc.empty() ? "__fmul2_rn(" + uu + ", " + k + ")" : "__ffma2_rn(" + uu + ", " + k + ", " + acc + ")";
                e.fma += (ca != 0.0) + (cb != 0.0);     // the useful products (the kernel's FMA count)
            }
            const std::string pn = pe.pre + "P" + std::to_string(pr.first) + "_" + std::to_string(pr.second);
            body << "    const float2 " << pn << " = " << acc << ";\n";
            body << "    const float " << mono_name(pr.first) << " = " << pn << ".x;\n";
            body << "    const float " << mono_name(pr.second) << " = " << pn << ".y;\n";
            pe.aname[r.mono[pr.first]] = mono_name(pr.first);
            pe.aname[r.mono[pr.second]] = mono_name(pr.second);
        }
        if (!kv.empty()) {
            std::ostringstream tab;
            for (size_t i = 0; i < kv.size(); ++i)
                tab << (i ? ", " : "") << "{" << flit(kv[i].first) << ", " << flit(kv[i].second) << "}";
            std::string name;
            auto it = e.kname_of.find(tab.str());
            if (it != e.kname_of.end()) {
                name = it->second;
            } else {
                name = "ls_K2_" + std::to_string(e.kname_of.size());
                e.kname_of[tab.str()] = name;
                e.ktabs += "__constant__ float2 " + name + "[" + std::to_string(kv.size()) + "] = {" + tab.str() +
                           "};\n";
            }
            std::string b = body.str(), out;
            for (size_t i = 0; i < b.size(); ++i) {
                if (b.compare(i, 2, "@K") == 0) out += name, i += 1;
                else out += b[i];
            }
            o << out;
        }
    }
    for (size_t a = 0; a < na; ++a) {
        if (partner[a] >= 0) continue;
        std::string acc;
        for (int v : f.live) {
            const double c = f.rows[(size_t)v][a];
            if (c == 0.0) continue;
            acc = acc.empty() ? flit(c) + " * " + vname(v) : "fmaf(" + flit(c) + ", " + vname(v) + ", " + acc + ")";
            e.fma++;
        }
        if (acc.empty()) continue;
        const std::string nm = mono_name(a);
        o << "    const float " << nm << " = " << acc << ";\n";
        pe.aname[r.mono[a]] = nm;
    }
}

// Emits value (and optionally gradient in reference coordinates) for region k.
// Returns names {f, g0, g1, g2}.
// Hessian entries in the order (0,0) (1,1) (2,2) (0,1) (0,2) (1,2) in 3D, (0,0) (1,1) (0,1) in 2D.
const int HI3[6] = {0, 1, 2, 0, 0, 1}, HJ3[6] = {0, 1, 2, 1, 2, 2};
const int HI2[3] = {0, 1, 0}, HJ2[3] = {0, 1, 1};

// Value, and for nd >= 1 the gradient, for nd >= 2 also the Hessian, all in
// reference coordinates: returns {f, g_0..g_{D-1}, h_0..h_{NH-1}}.
std::vector<std::string> emit_region_poly(Emitter &e, const Table &t, int k, const std::vector<int> &umap,
                                          int grad, const std::map<I3, std::string> *pre = nullptr)
{
    const RefRegion &r = t.ref[k];
    const int D = t.dim;
    PolyEmit pe{e, D, "r" + std::to_string(k) + "_", {}, {}, {}};
    if (pre) pe.aname = *pre;     // coefficients A_a computed elsewhere (tensor-core transform)
    for (int i = 0; i < D; ++i) {
        pe.uvar[i] = "u" + std::to_string(k) + "_" + std::to_string(i);
        e.o << "    const float " << pe.uvar[i] << " = a" << i << " - " << flit(r.center[i]) << ";\n";
    }
    std::set<I3> sup = monomial_support(r, umap, pe.terms);
    if (!pre && e.sym) {
        const FactoredTransform ft = factor_transform(r);
        if (!ft.ops.empty()) emit_factored_transform(e, r, umap, ft, pe);
    }
    // emit all A_a in a fixed order first (shared by value and gradient)
    for (const auto &m : sup) pe.A(m);
    auto coefA = [&](const I3 &m) -> std::string {
        auto it = pe.aname.find(m);
        return it == pe.aname.end() ? std::string() : it->second;
    };
    std::vector<std::string> res;
    std::string f = pe.horner(0, I3{0, 0, 0}, coefA, sup);
    res.push_back(f.empty() ? "0.0f" : f);
    if (grad) {
        for (int i = 0; i < D; ++i) {
            // derivative support and coefficients (ex_i + 1) * A_{m + e_i}
            std::set<I3> dsup;
            std::map<I3, std::string> dname;
            for (const auto &m : sup) {
                if (m[i] == 0) continue;
                I3 dm = m;
                dm[i] -= 1;
                dsup.insert(dm);
                std::string nm;
                if (m[i] == 1) {
                    nm = pe.aname[m];
                } else {
                    nm = e.fresh("dA");
                    e.o << "    const float " << nm << " = " << flit(m[i]) << " * " << pe.aname[m] << ";\n";
                    e.fma++;
                }
                dname[dm] = nm;
            }
            auto coefD = [&](const I3 &m) -> std::string {
                auto it = dname.find(m);
                return it == dname.end() ? std::string() : it->second;
            };
            std::string g = pe.horner(0, I3{0, 0, 0}, coefD, dsup);
            res.push_back(g.empty() ? "0.0f" : g);
        }
    }
    if (grad >= 2) {
        const int NH = D == 3 ? 6 : 3;
        for (int q = 0; q < NH; ++q) {
            const int i = D == 3 ? HI3[q] : HI2[q], j = D == 3 ? HJ3[q] : HJ2[q];
            // d^2/du_i du_j u^m = m_i (m_i - 1) u^{m - 2e_i} (i = j), m_i m_j u^{m - e_i - e_j} (i != j)
            std::set<I3> hsup;
            std::map<I3, std::string> hname;
            for (const auto &m : sup) {
                const int fac = (i == j) ? m[i] * (m[i] - 1) : m[i] * m[j];
                if (fac == 0) continue;
                I3 dm = m;
                dm[i] -= 1;
                dm[j] -= 1;
                hsup.insert(dm);
                std::string nm;
                if (fac == 1) {
                    nm = pe.aname[m];
                } else {
                    nm = e.fresh("hA");
                    e.o << "    const float " << nm << " = " << flit(fac) << " * " << pe.aname[m] << ";\n";
                    e.fma++;
                }
                hname[dm] = nm;
            }
            auto coefH = [&](const I3 &m) -> std::string {
                auto it = hname.find(m);
                return it == hname.end() ? std::string() : it->second;
            };
            std::string h = pe.horner(0, I3{0, 0, 0}, coefH, hsup);
            res.push_back(h.empty() ? "0.0f" : h);
        }
    }
    return res;
}

// Separable tensor-product evaluation (fold none, parallelepiped ROE).
// Emits value and optionally gradient; gathers are emitted here.
// Value, gradient and Hessian of a tensor-product spline: per-axis weights and
// their first and second derivatives, the gathers, then factorised sums
// sum_j2 W2 sum_j1 W1 sum_j0 W0 c for each derivative pattern (orders 0-2 per
// axis, total at most 2).
void emit_separable_hess(Emitter &e, const Table &t, std::string &fval, std::string g[3], std::string h[6])
{
    auto &o = e.o;
    const int D = t.dim;
    for (int i = 0; i < D; ++i) {
        const Axis &ax = t.sep[i];
        o << "    const float su" << i << " = y" << i << " - " << flit(ax.center) << ";\n";
        const int nc = ax.degree + 1;
        for (size_t j = 0; j < ax.sites.size(); ++j) {
            for (int der = 0; der <= 2; ++der) {
                // d^der/du^der of sum_d coef[d] u^d by Horner
                std::string acc;
                for (int d = ax.degree; d >= der; --d) {
                    double fac = 1.0;
                    for (int q = 0; q < der; ++q) fac *= (double)(d - q);
                    const std::string c = flit(ax.coef[j * nc + d] * fac);
                    if (acc.empty()) acc = c;
                    else {
                        acc = "fmaf(" + acc + ", su" + std::to_string(i) + ", " + c + ")";
                        e.fma++;
                    }
                }
                if (acc.empty()) acc = "0.0f";
                o << "    const float w" << der << "_" << i << "_" << j << " = " << acc << ";\n";
            }
        }
    }
    const int n[3] = {(int)t.sep[0].sites.size(), D > 1 ? (int)t.sep[1].sites.size() : 1,
                      D > 2 ? (int)t.sep[2].sites.size() : 1};
    std::vector<I3> sites;
    for (int j2 = 0; j2 < n[2]; ++j2)
        for (int j1 = 0; j1 < n[1]; ++j1)
            for (int j0 = 0; j0 < n[0]; ++j0)
                sites.push_back({t.sep[0].sites[j0], D > 1 ? t.sep[1].sites[j1] : 0, D > 2 ? t.sep[2].sites[j2] : 0});
    int reach = 0;
    for (auto &sv : sites)
        for (int i = 0; i < D; ++i) reach = std::max(reach, std::abs(sv[i]));
    emit_gathers(e, t, sites, reach, "a.coef", false, true, 0, 0);
    auto cidx = [&](int j0, int j1, int j2) { return (j2 * n[1] + j1) * n[0] + j0; };
    // derivative patterns (d0, d1, d2): f, g, h in output order
    std::vector<I3> pats = {{0, 0, 0}};
    for (int i = 0; i < D; ++i) { I3 p{0, 0, 0}; p[i] = 1; pats.push_back(p); }
    const int NH = D == 3 ? 6 : 3;
    for (int q = 0; q < NH; ++q) {
        const int i = D == 3 ? HI3[q] : HI2[q], j = D == 3 ? HJ3[q] : HJ2[q];
        I3 p{0, 0, 0};
        p[i] += 1;
        p[j] += 1;
        pats.push_back(p);
    }
    std::map<std::pair<int, int>, bool> t01;        // (d0, d1) partial sums needed
    std::map<int, bool> t0;
    for (auto &p : pats) { t0[p[0]] = true; t01[{p[0], p[1]}] = true; }
    for (auto &kv : t0) {
        const int d0 = kv.first;
        for (int j2 = 0; j2 < n[2]; ++j2)
            for (int j1 = 0; j1 < n[1]; ++j1) {
                std::string acc;
                for (int j0 = 0; j0 < n[0]; ++j0) {
                    const std::string term = "w" + std::to_string(d0) + "_0_" + std::to_string(j0);
                    const std::string c = "c" + std::to_string(cidx(j0, j1, j2));
                    acc = acc.empty() ? term + " * " + c : "fmaf(" + term + ", " + c + ", " + acc + ")";
                    e.fma++;
                }
                o << "    const float T" << d0 << "_" << j1 << "_" << j2 << " = " << acc << ";\n";
            }
    }
    std::map<std::pair<int, int>, std::vector<std::string>> U;
    for (auto &kv : t01) {
        const int d0 = kv.first.first, d1 = kv.first.second;
        for (int j2 = 0; j2 < n[2]; ++j2) {
            std::string acc;
            for (int j1 = 0; j1 < n[1]; ++j1) {
                const std::string tn = "T" + std::to_string(d0) + "_" + std::to_string(j1) + "_" + std::to_string(j2);
                if (D == 1) { acc = tn; break; }
                const std::string term = "w" + std::to_string(d1) + "_1_" + std::to_string(j1);
                acc = acc.empty() ? term + " * " + tn : "fmaf(" + term + ", " + tn + ", " + acc + ")";
                e.fma++;
            }
            std::string nm = "U" + std::to_string(d0) + std::to_string(d1) + "_" + std::to_string(j2);
            o << "    const float " << nm << " = " << acc << ";\n";
            U[{d0, d1}].push_back(nm);
        }
    }
    std::vector<std::string> outs;
    for (auto &p : pats) {
        const auto &uv = U[{p[0], p[1]}];
        std::string acc;
        if (D == 2) {
            acc = uv[0];
        } else {
            for (int j2 = 0; j2 < n[2]; ++j2) {
                const std::string term = "w" + std::to_string(p[2]) + "_2_" + std::to_string(j2);
                acc = acc.empty() ? term + " * " + uv[j2] : "fmaf(" + term + ", " + uv[j2] + ", " + acc + ")";
                e.fma++;
            }
        }
        std::string nm = e.fresh("sh");
        o << "    const float " << nm << " = " << acc << ";\n";
        outs.push_back(nm);
    }
    fval = outs[0];
    for (int i = 0; i < D; ++i) g[i] = outs[1 + i];
    for (int q = 0; q < NH; ++q) h[q] = outs[1 + D + q];
}

void emit_separable_body(Emitter &e, const Table &t, int grad, std::string &fval, std::string g[3],
                         std::string *h = nullptr)
{
    auto &o = e.o;
    const int D = t.dim;
    if (grad >= 2) {
        emit_separable_hess(e, t, fval, g, h);
        return;
    }
    // per-axis weights (and derivatives) by Horner in u = y - center
    for (int i = 0; i < D; ++i) {
        const Axis &ax = t.sep[i];
        o << "    const float su" << i << " = y" << i << " - " << flit(ax.center) << ";\n";
        const int nc = ax.degree + 1;
        for (size_t j = 0; j < ax.sites.size(); ++j) {
            std::string acc = flit(ax.coef[j * nc + ax.degree]);
            for (int d = ax.degree - 1; d >= 0; --d) {
                acc = "fmaf(" + acc + ", su" + std::to_string(i) + ", " + flit(ax.coef[j * nc + d]) + ")";
                e.fma++;
            }
            o << "    const float w" << i << "_" << j << " = " << acc << ";\n";
            if (grad) {
                std::string dacc = flit(ax.coef[j * nc + ax.degree] * ax.degree);
                for (int d = ax.degree - 1; d >= 1; --d) {
                    dacc = "fmaf(" + dacc + ", su" + std::to_string(i) + ", " + flit(ax.coef[j * nc + d] * d) + ")";
                    e.fma++;
                }
                o << "    const float dw" << i << "_" << j << " = " << dacc << ";\n";
            }
        }
    }
    const int n0 = (int)t.sep[0].sites.size(), n1 = D > 1 ? (int)t.sep[1].sites.size() : 1,
              n2 = D > 2 ? (int)t.sep[2].sites.size() : 1;
    // gathers in rows along axis 0
    std::vector<I3> sites;
    for (int j2 = 0; j2 < n2; ++j2)
        for (int j1 = 0; j1 < n1; ++j1)
            for (int j0 = 0; j0 < n0; ++j0)
                sites.push_back({t.sep[0].sites[j0], D > 1 ? t.sep[1].sites[j1] : 0, D > 2 ? t.sep[2].sites[j2] : 0});
    int reach = 0;
    for (auto &s : sites)
        for (int i = 0; i < D; ++i) reach = std::max(reach, std::abs(s[i]));
    emit_gathers(e, t, sites, reach, "a.coef", false);
    auto cidx = [&](int j0, int j1, int j2) { return (j2 * n1 + j1) * n0 + j0; };
    // contraction along axis 0: T(j1,j2) = sum w0 c ; dT = sum dw0 c
    for (int j2 = 0; j2 < n2; ++j2)
        for (int j1 = 0; j1 < n1; ++j1) {
            std::string acc = "w0_0 * c" + std::to_string(cidx(0, j1, j2));
            std::string dacc = "dw0_0 * c" + std::to_string(cidx(0, j1, j2));
            e.fma += grad ? 2 : 1;
            for (int j0 = 1; j0 < n0; ++j0) {
                acc = "fmaf(w0_" + std::to_string(j0) + ", c" + std::to_string(cidx(j0, j1, j2)) + ", " + acc + ")";
                dacc = "fmaf(dw0_" + std::to_string(j0) + ", c" + std::to_string(cidx(j0, j1, j2)) + ", " + dacc + ")";
                e.fma += grad ? 2 : 1;
            }
            o << "    const float T" << j1 << "_" << j2 << " = " << acc << ";\n";
            if (grad) o << "    const float dT" << j1 << "_" << j2 << " = " << dacc << ";\n";
        }
    if (D == 2) {
        std::string f = "0.0f", g0 = "0.0f", g1 = "0.0f";
        for (int j1 = 0; j1 < n1; ++j1) {
            std::string s1 = std::to_string(j1);
            f = "fmaf(w1_" + s1 + ", T" + s1 + "_0, " + f + ")";
            e.fma++;
            if (grad) {
                g0 = "fmaf(w1_" + s1 + ", dT" + s1 + "_0, " + g0 + ")";
                g1 = "fmaf(dw1_" + s1 + ", T" + s1 + "_0, " + g1 + ")";
                e.fma += 2;
            }
        }
        o << "    const float fv = " << f << ";\n";
        fval = "fv";
        if (grad) {
            o << "    const float gr0 = " << g0 << ";\n    const float gr1 = " << g1 << ";\n";
            g[0] = "gr0";
            g[1] = "gr1";
        }
        return;
    }
    // axis 1: U(j2) = sum w1 T, U1(j2) = sum dw1 T, V(j2) = sum w1 dT
    for (int j2 = 0; j2 < n2; ++j2) {
        std::string u = "0.0f", u1 = "0.0f", v = "0.0f";
        for (int j1 = 0; j1 < n1; ++j1) {
            std::string tn = "T" + std::to_string(j1) + "_" + std::to_string(j2);
            u = "fmaf(w1_" + std::to_string(j1) + ", " + tn + ", " + u + ")";
            e.fma++;
            if (grad) {
                u1 = "fmaf(dw1_" + std::to_string(j1) + ", " + tn + ", " + u1 + ")";
                v = "fmaf(w1_" + std::to_string(j1) + ", d" + tn + ", " + v + ")";
                e.fma += 2;
            }
        }
        o << "    const float U" << j2 << " = " << u << ";\n";
        if (grad) o << "    const float U1_" << j2 << " = " << u1 << ";\n    const float V" << j2 << " = " << v << ";\n";
    }
    std::string f = "0.0f", g0 = "0.0f", g1 = "0.0f", g2 = "0.0f";
    for (int j2 = 0; j2 < n2; ++j2) {
        std::string s2 = std::to_string(j2);
        f = "fmaf(w2_" + s2 + ", U" + s2 + ", " + f + ")";
        e.fma++;
        if (grad) {
            g0 = "fmaf(w2_" + s2 + ", V" + s2 + ", " + g0 + ")";
            g1 = "fmaf(w2_" + s2 + ", U1_" + s2 + ", " + g1 + ")";
            g2 = "fmaf(dw2_" + s2 + ", U" + s2 + ", " + g2 + ")";
            e.fma += 3;
        }
    }
    o << "    const float fv = " << f << ";\n";
    fval = "fv";
    if (grad) {
        o << "    const float gr0 = " << g0 << ";\n    const float gr1 = " << g1 << ";\n    const float gr2 = " << g2
          << ";\n";
        g[0] = "gr0";
        g[1] = "gr1";
        g[2] = "gr2";
    }
}

// Out-of-range and NaN coordinates: zero (NaN for NaN) instead of a value.
void emit_point_check(Emitter &e, const Table &t, const char *skip)
{
    auto &o = e.o;
    const int D = t.dim;
    o << "    if (!(";
    for (int i = 0; i < D; ++i) o << (i ? " && " : "") << "fabsf(x" << i << ") < 4194304.0f";
    o << ")) {\n";
    o << "      const bool isn = ";
    for (int i = 0; i < D; ++i) o << (i ? " || " : "") << "(x" << i << " != x" << i << ")";
    o << ";\n";
    o << "      LS_OUT_OF_RANGE(isn ? __int_as_float(0x7fffffff) : 0.0f);\n";
    o << "      " << skip << ";\n    }\n";
}

void emit_point_load(Emitter &e, const Table &t, const char *skip = "continue")
{
    auto &o = e.o;
    const int D = t.dim;
    for (int i = 0; i < D; ++i)
        o << "    const float x" << i << " = ls_ld_pt(a.pts + (size_t)i * " << D << " + " << i << ");\n";
    emit_point_check(e, t, skip);
}

std::string kname(const Table &t, const char *what)
{
    std::string n = "ls_" + std::string(what);
    if (!t.name.empty()) n += "__" + t.name;
    return n;
}

// Per-point evaluation of value [+ gradient] as a device function, reused by
// the per-spline kernel and by batched (multi-volume) kernels.
void emit_eval_point(Emitter &e, const Table &t, const ls_variant &var, const Stencil &st, int reach, bool grad,
                     const std::string &fname, bool coords_args = false, bool check = false)
{
    auto &o = e.o;
    const int D = t.dim;
    if (coords_args)
        // the point is given (finite, in range): used by the staged kernel with
        // coordinates relative to its tile
        o << "static __device__ __forceinline__ void " << fname
          << "(const LsEvalArgs& a, const long long i, const float x0, const float x1, const float x2)\n{\n"
             "  (void)x2;\n";
    else
        o << "static __device__ __forceinline__ void " << fname << "(const LsEvalArgs& a, const long long i)\n{\n";
    o << "  const int E0 = a.e0, E1 = a.e1, E2 = a.e2, CS = a.cstride, CU = a.cunit;"
         " (void)E1; (void)E2; (void)CS; (void)CU;\n";
    if (grad) {
        o << "#define LS_OUT_OF_RANGE(V) { if (a.out) a.out[i] = (V);";
        for (int i = 0; i < D; ++i) o << " a.grad[(size_t)i * " << D << " + " << i << "] = (V);";
        o << " }\n";
    } else {
        o << "#define LS_OUT_OF_RANGE(V) { a.out[i] = (V); }\n";
    }
    o << "  {\n";
    if (!coords_args) emit_point_load(e, t, "return");
    else if (check) emit_point_check(e, t, "return");
    emit_classify(e, t);
    std::string fv;
    std::string g[3];
    if (!t.sep.empty()) {
        emit_separable_body(e, t, grad, fv, g);
    } else {
        emit_gathers(e, t, st.sites, reach, "a.coef", false, true, var.group, var.depth);
        const size_t K = t.ref.size();
        std::vector<std::vector<std::string>> rr;
        if (K > 1 && var.branchy) {
            o << "    float fsel = 0.0f, gs0 = 0.0f, gs1 = 0.0f, gs2 = 0.0f;\n";
            for (size_t k = 0; k < K; ++k) {
                o << "    " << (k ? "else " : "") << "if (psi == " << k << ") {\n";
                auto r = emit_region_poly(e, t, (int)k, st.region_to_union[k], grad);
                o << "    fsel = " << r[0] << ";\n";
                if (grad)
                    for (int i = 0; i < D; ++i) o << "    gs" << i << " = " << r[1 + i] << ";\n";
                o << "    }\n";
            }
            fv = "fsel";
            for (int i = 0; i < D; ++i) g[i] = "gs" + std::to_string(i);
        } else {
            for (size_t k = 0; k < K; ++k) rr.push_back(emit_region_poly(e, t, (int)k, st.region_to_union[k], grad));
            if (K == 1) {
                fv = rr[0][0];
                if (grad)
                    for (int i = 0; i < D; ++i) g[i] = rr[0][1 + i];
            } else {
                for (int c = 0; c < (grad ? D + 1 : 1); ++c) {
                    std::string sel = rr[K - 1][c];
                    for (int k = (int)K - 2; k >= 0; --k)
                        sel = "(psi == " + std::to_string(k) + ") ? " + rr[k][c] + " : (" + sel + ")";
                    std::string nm = c == 0 ? "fsel" : "gs" + std::to_string(c - 1);
                    o << "    const float " << nm << " = " << sel << ";\n";
                }
                fv = "fsel";
                for (int i = 0; i < D; ++i) g[i] = "gs" + std::to_string(i);
            }
        }
    }
    if (grad) {
        o << "    if (a.out) ls_st_out(a.out + i, " << fv << ");\n";
        // chain rule back to Cartesian axes: df/dy_i = sign_i * g[ref axis landing on i]
        for (int i = 0; i < D; ++i) {
            if (t.fold == LS_FOLD_SIGNED_PERM) {
                o << "    { const float gg = ";
                for (int r = 0; r < D - 1; ++r) o << "(ri" << i << " == " << r << ") ? " << g[r] << " : ";
                o << g[D - 1] << "; ls_st_out(a.grad + (size_t)i * " << D << " + " << i << ", ng" << i << " ? -gg : gg); }\n";
            } else {
                o << "    ls_st_out(a.grad + (size_t)i * " << D << " + " << i << ", " << g[i] << ");\n";
            }
        }
    } else {
        o << "    ls_st_out(a.out + i, " << fv << ");\n";
    }
    o << "  }\n#undef LS_OUT_OF_RANGE\n}\n\n";
}

// Value, gradient and Hessian at one point (Sec. 3: the derivatives of the
// per-region polynomials; symmetry still applies).  In the folded frame the
// Hessian of f is H_ref; on Cartesian axes a, b it is
//     H[a][b] = s_a s_b H_ref[r(a)][r(b)]
// with r(a) the reference axis that lands on axis a and s_a its sign.  Output
// a.hess[i * NH + q] in the order xx yy zz xy xz yz (2D: xx yy xy); a.out and
// a.grad may be null.
void emit_eval_point_hess(Emitter &e, const Table &t, const ls_variant &var, const Stencil &st, int reach,
                          const std::string &fname)
{
    auto &o = e.o;
    const int D = t.dim;
    const int NH = D == 3 ? 6 : 3;
    const int NO = 1 + D + NH;
    o << "static __device__ __forceinline__ void " << fname << "(const LsEvalArgs& a, const long long i)\n{\n";
    o << "  const int E0 = a.e0, E1 = a.e1, E2 = a.e2, CS = a.cstride, CU = a.cunit;"
         " (void)E1; (void)E2; (void)CS; (void)CU;\n";
    o << "#define LS_OUT_OF_RANGE(V) { if (a.out) a.out[i] = (V); if (a.grad) {";
    for (int i = 0; i < D; ++i) o << " a.grad[(size_t)i * " << D << " + " << i << "] = (V);";
    o << " }";
    for (int q = 0; q < NH; ++q) o << " a.hess[(size_t)i * " << NH << " + " << q << "] = (V);";
    o << " }\n";
    o << "  {\n";
    emit_point_load(e, t, "return");
    emit_classify(e, t);
    std::vector<std::string> res(NO);
    if (!t.sep.empty()) {
        std::string g[3], h[6];
        emit_separable_body(e, t, 2, res[0], g, h);
        for (int i = 0; i < D; ++i) res[1 + i] = g[i];
        for (int q = 0; q < NH; ++q) res[1 + D + q] = h[q];
    } else {
        emit_gathers(e, t, st.sites, reach, "a.coef", false, true, 0, 0);
        const size_t K = t.ref.size();
        if (K > 1 && var.branchy) {
            for (int c = 0; c < NO; ++c) o << "    float hs" << c << " = 0.0f;\n";
            for (size_t k = 0; k < K; ++k) {
                o << "    " << (k ? "else " : "") << "if (psi == " << k << ") {\n";
                auto r = emit_region_poly(e, t, (int)k, st.region_to_union[k], 2);
                for (int c = 0; c < NO; ++c) o << "    hs" << c << " = " << r[c] << ";\n";
                o << "    }\n";
            }
            for (int c = 0; c < NO; ++c) res[c] = "hs" + std::to_string(c);
        } else {
            std::vector<std::vector<std::string>> rr;
            for (size_t k = 0; k < K; ++k) rr.push_back(emit_region_poly(e, t, (int)k, st.region_to_union[k], 2));
            for (int c = 0; c < NO; ++c) {
                std::string sel = rr[K - 1][c];
                for (int k = (int)K - 2; k >= 0; --k)
                    sel = "(psi == " + std::to_string(k) + ") ? " + rr[k][c] + " : (" + sel + ")";
                o << "    const float hs" << c << " = " << sel << ";\n";
                res[c] = "hs" + std::to_string(c);
            }
        }
    }
    o << "    if (a.out) ls_st_out(a.out + i, " << res[0] << ");\n";
    const bool fold = t.fold == LS_FOLD_SIGNED_PERM;
    o << "    if (a.grad) {\n";
    for (int i = 0; i < D; ++i) {
        if (fold) {
            o << "    { const float gg = ";
            for (int r = 0; r < D - 1; ++r) o << "(ri" << i << " == " << r << ") ? " << res[1 + r] << " : ";
            o << res[1 + D - 1] << "; ls_st_out(a.grad + (size_t)i * " << D << " + " << i << ", ng" << i << " ? -gg : gg); }\n";
        } else {
            o << "    ls_st_out(a.grad + (size_t)i * " << D << " + " << i << ", " << res[1 + i] << ");\n";
        }
    }
    o << "    }\n";
    // reference Hessian entry of reference axes (r1, r2)
    auto href = [&](int r1, int r2) {
        if (r1 > r2) std::swap(r1, r2);
        for (int q = 0; q < NH; ++q) {
            const int qi = D == 3 ? HI3[q] : HI2[q], qj = D == 3 ? HJ3[q] : HJ2[q];
            if (qi == r1 && qj == r2) return res[1 + D + q];
        }
        return std::string("0.0f");
    };
    for (int q = 0; q < NH; ++q) {
        const int ca = D == 3 ? HI3[q] : HI2[q], cb = D == 3 ? HJ3[q] : HJ2[q];
        if (fold) {
            std::string sel;
            for (int r1 = D - 1; r1 >= 0; --r1) {
                std::string inner;
                for (int r2 = D - 1; r2 >= 0; --r2)
                    inner = inner.empty() ? href(r1, r2)
                                          : "(ri" + std::to_string(cb) + " == " + std::to_string(r2) + ") ? " +
                                                href(r1, r2) + " : (" + inner + ")";
                sel = sel.empty() ? inner
                                  : "(ri" + std::to_string(ca) + " == " + std::to_string(r1) + ") ? (" + inner +
                                        ") : (" + sel + ")";
            }
            o << "    { const float hh = " << sel << "; ls_st_out(a.hess + (size_t)i * " << NH << " + " << q << ", (ng" << ca
              << " ^ ng" << cb << ") ? -hh : hh); }\n";
        } else {
            o << "    ls_st_out(a.hess + (size_t)i * " << NH << " + " << q << ", " << href(ca, cb) << ");\n";
        }
    }
    o << "  }\n#undef LS_OUT_OF_RANGE\n}\n\n";
}

// Coherent-reuse evaluation kernel: each thread walks T consecutive points and
// repeats the gathers and the coefficient transform A = M c only when the
// region-of-evaluation site, the fold transform or the reference sub-region
// changes; the Horner form runs per point.  For ray-ordered points most
// neighbours share them.  Results equal the one-point-per-thread kernel.
void emit_eval_kernel_reuse(Emitter &e, const Table &t, const ls_variant &var, const Stencil &st, int reach,
                            int T, GenInfo &info)
{
    auto &o = e.o;
    const int D = t.dim;
    const int fma0 = e.fma;
    const size_t K = t.ref.size();
    // monomial supports and A names per region
    std::vector<std::map<I3, std::vector<std::pair<int, double>>>> terms(K);
    std::vector<std::set<I3>> sup(K);
    for (size_t k = 0; k < K; ++k) sup[k] = monomial_support(t.ref[k], st.region_to_union[k], terms[k]);
    auto aname = [&](size_t k, const I3 &m) {
        return "r" + std::to_string(k) + "_A" + std::to_string(m[0]) + "_" + std::to_string(m[1]) + "_" +
               std::to_string(m[2]);
    };
    o << "extern \"C\" __global__ void __launch_bounds__(" << var.block;
    if (var.min_blocks > 0) o << ", " << var.min_blocks;
    o << ") " << kname(t, "eval") << "(const LsEvalArgs a)\n{\n";
    o << "  const int E0 = a.e0, E1 = a.e1, E2 = a.e2, CS = a.cstride, CU = a.cunit;"
         " (void)E1; (void)E2; (void)CS; (void)CU;\n";
    o << "  const long long nchunk = (a.n + " << T - 1 << ") / " << T << ";\n";
    o << "  const long long cstride_ = (long long)gridDim.x * blockDim.x;\n";
    o << "#define LS_OUT_OF_RANGE(V) { a.out[i] = (V); }\n";
    o << "  for (long long ch = (long long)blockIdx.x * blockDim.x + threadIdx.x; ch < nchunk; ch += cstride_) {\n";
    for (size_t k = 0; k < K; ++k)
        for (const auto &m : sup[k]) o << "    float " << aname(k, m) << " = 0.0f;\n";
    o << "    int pk0 = 0x7fffffff, pk1 = 0, pk2 = 0, pcode = -1, ppsi = -1;\n";
    o << "    const long long iend = (ch + 1) * " << T << " < a.n ? (ch + 1) * " << T << " : a.n;\n";
    o << "    for (long long i = ch * " << T << "; i < iend; ++i) {\n";
    emit_point_load(e, t, "continue");
    emit_classify(e, t);
    if (t.fold == LS_FOLD_SIGNED_PERM)
        o << "    const int code = p0 | (p1 << 2) | ((int)g0 << 4)" << (D > 1 ? " | ((int)g1 << 5)" : "")
          << (D > 2 ? " | ((int)g2 << 6)" : "") << ";\n";
    else
        o << "    const int code = 0;\n";
    o << "    const bool same = (k0 == pk0)" << (D > 1 ? " && (k1 == pk1)" : "") << (D > 2 ? " && (k2 == pk2)" : "")
      << " && (code == pcode) && (psi == ppsi);\n";
    o << "    if (!same) {\n";
    emit_gathers(e, t, st.sites, reach, "a.coef", false);
    for (size_t k = 0; k < K; ++k) {
        // the same transform as the one-point kernel (factored when the
        // generator factors it), so the results stay bit for bit the same
        const FactoredTransform ft = e.sym ? factor_transform(t.ref[k]) : FactoredTransform();
        if (!ft.ops.empty()) {
            PolyEmit pe{e, D, "t" + std::to_string(k) + "_", {}, {}, {}};
            o << "    {\n";
            emit_factored_transform(e, t.ref[k], st.region_to_union[k], ft, pe);
            for (const auto &m : sup[k]) o << "    " << aname(k, m) << " = " << pe.aname[m] << ";\n";
            o << "    }\n";
            continue;
        }
        for (const auto &m : sup[k]) {
            std::string acc;
            for (auto &pr : terms[k][m]) {
                acc = acc.empty() ? flit(pr.second) + " * c" + std::to_string(pr.first)
                                  : "fmaf(" + flit(pr.second) + ", c" + std::to_string(pr.first) + ", " + acc + ")";
                e.fma++;
            }
            o << "    " << aname(k, m) << " = " << acc << ";\n";
        }
    }
    o << "    pk0 = k0;" << (D > 1 ? " pk1 = k1;" : "") << (D > 2 ? " pk2 = k2;" : "") << " pcode = code; ppsi = psi;\n";
    o << "    }\n";
    std::vector<std::string> fk;
    for (size_t k = 0; k < K; ++k) {
        PolyEmit pe{e, D, "", {}, {}, {}};
        for (int i = 0; i < D; ++i) {
            pe.uvar[i] = "u" + std::to_string(k) + "_" + std::to_string(i);
            o << "    const float " << pe.uvar[i] << " = a" << i << " - " << flit(t.ref[k].center[i]) << ";\n";
        }
        auto coefA = [&](const I3 &m) -> std::string { return sup[k].count(m) ? aname(k, m) : std::string(); };
        std::string f = pe.horner(0, I3{0, 0, 0}, coefA, sup[k]);
        fk.push_back(f.empty() ? "0.0f" : f);
    }
    std::string sel = fk[K - 1];
    for (int k = (int)K - 2; k >= 0; --k) sel = "(psi == " + std::to_string(k) + ") ? " + fk[k] + " : (" + sel + ")";
    o << "    ls_st_out(a.out + i, " << sel << ");\n";
    o << "    }\n  }\n#undef LS_OUT_OF_RANGE\n}\n\n";
    info.fma_value = e.fma - fma0;
}

// value [+ gradient] kernel: grid-stride loop over the point function
void emit_eval_kernel(Emitter &e, const Table &t, const ls_variant &var, const Stencil &st, int reach,
                      bool grad, GenInfo &info)
{
    auto &o = e.o;
    const int fma0 = e.fma;
    const std::string pf = kname(t, grad ? "eval_grad_pt" : "eval_pt");
    const int D = t.dim;
    if (var.prefetch) {
        // the coordinates of a thread's next point are loaded before the current
        // point is evaluated, so their latency (HBM: the points stream through)
        // is off the path of the gathers
        emit_eval_point(e, t, var, st, reach, grad, pf + "_x", true, true);
        o << "extern \"C\" __global__ void __launch_bounds__(" << var.block;
        if (var.min_blocks > 0) o << ", " << var.min_blocks;
        o << ") " << kname(t, grad ? "eval_grad" : "eval") << "(const LsEvalArgs a)\n{\n";
        o << "  const long long stride = (long long)gridDim.x * blockDim.x;\n";
        o << "  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;\n";
        o << "  float n0 = 0.0f, n1 = 0.0f, n2 = 0.0f;\n";
        o << "  if (i < a.n) {";
        for (int q = 0; q < D; ++q) o << " n" << q << " = ls_ld_pt(a.pts + (size_t)i * " << D << " + " << q << ");";
        o << " }\n";
        o << "  for (; i < a.n; i += stride) {\n";
        o << "    const float x0 = n0, x1 = n1, x2 = n2;\n";
        o << "    if (i + stride < a.n) {";
        for (int q = 0; q < D; ++q)
            o << " n" << q << " = ls_ld_pt(a.pts + (size_t)(i + stride) * " << D << " + " << q << ");";
        o << " }\n";
        o << "    " << pf << "_x(a, i, x0, x1, x2);\n  }\n}\n\n";
    } else {
        emit_eval_point(e, t, var, st, reach, grad, pf);
        o << "extern \"C\" __global__ void __launch_bounds__(" << var.block;
        if (var.min_blocks > 0) o << ", " << var.min_blocks;
        o << ") " << kname(t, grad ? "eval_grad" : "eval") << "(const LsEvalArgs a)\n{\n";
        o << "  const long long stride = (long long)gridDim.x * blockDim.x;\n";
        o << "  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) " << pf
          << "(a, i);\n}\n\n";
    }
    if (grad) info.fma_grad = e.fma - fma0;
    else info.fma_value = e.fma - fma0;
}

// Software-pipelined value kernel: every thread keeps the gathers of its next
// point in flight while it evaluates the polynomial of the current one (two
// point states P and Q, alternating), so a few warps per SM keep the L1 miss
// path busy while fewer stencils compete for L1.  Stage A: point load, region
// of evaluation, sub-region, gathers; stage B: polynomial and store.
void emit_eval_kernel_pipelined(Emitter &e, const Table &t, const ls_variant &var, const Stencil &st, int reach,
                                GenInfo &info)
{
    auto &o = e.o;
    const int D = t.dim;
    const size_t NS = st.sites.size();
    const size_t K = t.ref.size();
    auto stage_a = [&](const std::string &S, const std::string &idx) {
        o << "  {\n    const long long i = " << idx << ";\n";
        o << "    " << S << "_sp = 0;\n";
        o << "#define LS_OUT_OF_RANGE(V) { " << S << "_sp = 1; " << S << "_sv = (V); }\n";
        o << "    do {\n";
        emit_point_load(e, t, "break");
        emit_classify(e, t);
        emit_gathers(e, t, st.sites, reach, "a.coef", false, true, 0, 0);
        for (size_t j = 0; j < NS; ++j) o << "    " << S << "_c" << j << " = c" << j << ";\n";
        for (int i = 0; i < D; ++i) o << "    " << S << "_a" << i << " = a" << i << ";\n";
        o << "    " << S << "_psi = psi;\n";
        o << "    } while (0);\n#undef LS_OUT_OF_RANGE\n  }\n";
    };
    auto stage_b = [&](const std::string &S, const std::string &idx) {
        o << "  {\n";
        for (size_t j = 0; j < NS; ++j) o << "    const float c" << j << " = " << S << "_c" << j << ";\n";
        for (int i = 0; i < D; ++i) o << "    const float a" << i << " = " << S << "_a" << i << ";\n";
        o << "    const int psi = " << S << "_psi; (void)psi;\n";
        std::string fv;
        if (K > 1 && var.branchy) {
            o << "    float fsel = 0.0f;\n";
            for (size_t k = 0; k < K; ++k) {
                o << "    " << (k ? "else " : "") << "if (psi == " << k << ") {\n";
                auto r = emit_region_poly(e, t, (int)k, st.region_to_union[k], false);
                o << "    fsel = " << r[0] << ";\n    }\n";
            }
            fv = "fsel";
        } else {
            std::vector<std::string> rr;
            for (size_t k = 0; k < K; ++k) rr.push_back(emit_region_poly(e, t, (int)k, st.region_to_union[k], false)[0]);
            std::string sel = rr[K - 1];
            for (int k = (int)K - 2; k >= 0; --k) sel = "(psi == " + std::to_string(k) + ") ? " + rr[k] + " : (" + sel + ")";
            o << "    const float fsel = " << sel << ";\n";
            fv = "fsel";
        }
        o << "    a.out[" << idx << "] = " << S << "_sp ? " << S << "_sv : " << fv << ";\n  }\n";
    };
    o << "extern \"C\" __global__ void __launch_bounds__(" << var.block;
    if (var.min_blocks > 0) o << ", " << var.min_blocks;
    o << ") " << kname(t, "eval") << "(const LsEvalArgs a)\n{\n";
    o << "  const int E0 = a.e0, E1 = a.e1, E2 = a.e2, CS = a.cstride, CU = a.cunit;"
         " (void)E1; (void)E2; (void)CS; (void)CU;\n";
    o << "  const long long stride = (long long)gridDim.x * blockDim.x;\n";
    for (const char *S : {"P", "Q"}) {
        for (size_t j = 0; j < NS; ++j) o << "  float " << S << "_c" << j << " = 0.0f;\n";
        for (int i = 0; i < D; ++i) o << "  float " << S << "_a" << i << " = 0.0f;\n";
        o << "  int " << S << "_psi = 0, " << S << "_sp = 0; float " << S << "_sv = 0.0f;\n";
    }
    o << "  long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;\n";
    o << "  if (i0 >= a.n) return;\n";
    stage_a("P", "i0");
    o << "  for (;;) {\n";
    o << "  const long long i1 = i0 + stride;\n";
    o << "  if (i1 < a.n)\n";
    stage_a("Q", "i1");
    const int fma0 = e.fma;
    stage_b("P", "i0");
    info.fma_value = e.fma - fma0;
    o << "  if (i1 >= a.n) break;\n";
    o << "  i0 = i1 + stride;\n";
    o << "  if (i0 < a.n)\n";
    stage_a("P", "i0");
    stage_b("Q", "i1");
    o << "  if (i0 >= a.n) break;\n";
    o << "  }\n}\n\n";
}

// Warp-specialized value kernel.  The first P warps of a block (producers)
// classify points and gather their coefficients into shared-memory slots, one
// slot of 32 points per consumer warp; the other warps (consumers) evaluate the
// polynomials from the slots.  Few stencils are in flight per SM (P x 32
// points), so their cache lines stay in L1 between the gathers of one point,
// while many warps hide the latency of the polynomial.  Slot k has two
// mbarriers: full[k] (the producer's lane 0 arrives after the warp's stores)
// and empty[k] (the consumer's lane 0 arrives after the warp's loads); phases
// alternate per round.  Every wait is bounded: a wait that gives up sets
// *a.status and its warp leaves, so no warp can wait forever.
// Returns the dynamic shared-memory bytes of the kernel.
int emit_eval_kernel_ws(Emitter &e, const Table &t, const ls_variant &var, const Stencil &st, int reach,
                        GenInfo &info)
{
    auto &o = e.o;
    const int D = t.dim;
    const int NS = (int)st.sites.size();
    const size_t K = t.ref.size();
    const int NP = var.producers;
    const int NC = var.block / 32 - NP;
    const int SLOT = (NS + D + 2) * 32;          // floats: c[NS][32], a[D][32], meta (psi | flags), special value
    const int smem = NC * SLOT * 4 + 2 * NC * 8;
    o << "extern \"C\" __global__ void __launch_bounds__(" << var.block;
    if (var.min_blocks > 0) o << ", " << var.min_blocks;
    o << ") " << kname(t, "eval") << "(const LsEvalArgs a)\n{\n";
    o << "  extern __shared__ __align__(16) float ls_slots[];\n";
    o << "  const int E0 = a.e0, E1 = a.e1, E2 = a.e2, CS = a.cstride, CU = a.cunit;"
         " (void)E1; (void)E2; (void)CS; (void)CU;\n";
    o << "  const unsigned bar0 = (unsigned)__cvta_generic_to_shared(ls_slots + " << NC * SLOT << ");\n";
    o << "  // full[k] at bar0 + 8k, empty[k] at bar0 + 8(" << NC << " + k)\n";
    o << "  if (threadIdx.x == 0) {\n";
    o << "    for (int k = 0; k < " << 2 * NC << "; ++k)\n";
    o << "      asm volatile(\"mbarrier.init.shared::cta.b64 [%0], 1;\" :: \"r\"(bar0 + 8u * k) : \"memory\");\n";
    o << "  }\n  __syncthreads();\n";
    o << "  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;\n";
    o << "  const long long TILE = " << 32 * NC << "LL;\n";
    o << "  const long long ntiles = (a.n + TILE - 1) / TILE;\n";
    o << "  const long long rounds = ntiles > (long long)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;\n";
    // producers
    o << "  if (warp < " << NP << ") {\n";
    o << "    for (long long r = 0; r < rounds; ++r) {\n";
    o << "      const long long tile = (long long)blockIdx.x + r * gridDim.x;\n";
    o << "      for (int k = warp; k < " << NC << "; k += " << NP << ") {\n";
    o << "        if (r > 0 && !ls_mbar_wait(bar0 + 8u * (" << NC << " + k), (unsigned)((r - 1) & 1), a.status)) return;\n";
    o << "        float* sl = ls_slots + k * " << SLOT << ";\n";
    o << "        const long long i = tile * TILE + k * 32 + lane;\n";
    o << "        int sp = 0; float sv = 0.0f; int psi_out = 0;\n";
    for (int j = 0; j < NS; ++j) o << "        float oc" << j << " = 0.0f;\n";
    for (int i = 0; i < D; ++i) o << "        float oa" << i << " = 0.0f;\n";
    o << "#define LS_OUT_OF_RANGE(V) { sp = 1; sv = (V); }\n";
    o << "        do {\n";
    o << "        if (i >= a.n) { sp = 2; break; }\n";
    emit_point_load(e, t, "break");
    emit_classify(e, t);
    emit_gathers(e, t, st.sites, reach, "a.coef", false, true, 0, 0);
    for (int j = 0; j < NS; ++j) o << "        oc" << j << " = c" << j << ";\n";
    for (int i = 0; i < D; ++i) o << "        oa" << i << " = a" << i << ";\n";
    o << "        psi_out = psi;\n";
    o << "        } while (0);\n#undef LS_OUT_OF_RANGE\n";
    for (int j = 0; j < NS; ++j) o << "        sl[" << j * 32 << " + lane] = oc" << j << ";\n";
    for (int i = 0; i < D; ++i) o << "        sl[" << (NS + i) * 32 << " + lane] = oa" << i << ";\n";
    o << "        sl[" << (NS + D) * 32 << " + lane] = __int_as_float(psi_out | (sp << 8));\n";
    o << "        sl[" << (NS + D + 1) * 32 << " + lane] = sv;\n";
    o << "        __syncwarp();\n";
    if (e.no_signal)   // test hook: the slot is never signalled, so every consumer's wait runs out
        o << "        // (no arrival: wait_probe)\n";
    else
        o << "        if (lane == 0) asm volatile(\"mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\" :: \"r\"(bar0 + 8u * k) : \"memory\");\n";
    o << "      }\n    }\n    return;\n  }\n";
    // consumers
    o << "  {\n";
    o << "    const int k = warp - " << NP << ";\n";
    o << "    const float* sl = ls_slots + k * " << SLOT << ";\n";
    o << "    for (long long r = 0; r < rounds; ++r) {\n";
    o << "      const long long tile = (long long)blockIdx.x + r * gridDim.x;\n";
    o << "      const long long i = tile * TILE + k * 32 + lane;\n";
    o << "      if (!ls_mbar_wait(bar0 + 8u * k, (unsigned)(r & 1), a.status)) return;\n";
    for (int j = 0; j < NS; ++j) o << "      const float c" << j << " = sl[" << j * 32 << " + lane];\n";
    for (int i = 0; i < D; ++i) o << "      const float a" << i << " = sl[" << (NS + i) * 32 << " + lane];\n";
    o << "      const int meta = __float_as_int(sl[" << (NS + D) * 32 << " + lane]);\n";
    o << "      const float sv = sl[" << (NS + D + 1) * 32 << " + lane];\n";
    o << "      __syncwarp();\n";
    o << "      if (lane == 0) asm volatile(\"mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\" :: \"r\"(bar0 + 8u * ("
      << NC << " + k)) : \"memory\");\n";
    o << "      const int psi = meta & 255, sp = meta >> 8; (void)psi;\n";
    const int fma0 = e.fma;
    std::string fv;
    if (K > 1 && var.branchy) {
        o << "      float fsel = 0.0f;\n";
        for (size_t k = 0; k < K; ++k) {
            o << "      " << (k ? "else " : "") << "if (psi == " << k << ") {\n";
            auto r = emit_region_poly(e, t, (int)k, st.region_to_union[k], false);
            o << "      fsel = " << r[0] << ";\n      }\n";
        }
        fv = "fsel";
    } else {
        std::vector<std::string> rr;
        for (size_t k = 0; k < K; ++k) rr.push_back(emit_region_poly(e, t, (int)k, st.region_to_union[k], false)[0]);
        std::string sel = rr[K - 1];
        for (int k = (int)K - 2; k >= 0; --k) sel = "(psi == " + std::to_string(k) + ") ? " + rr[k] + " : (" + sel + ")";
        o << "      const float fsel = " << sel << ";\n";
        fv = "fsel";
    }
    info.fma_value = e.fma - fma0;
    o << "      if (sp != 2) a.out[i] = sp ? sv : " << fv << ";\n";
    o << "    }\n  }\n}\n\n";
    return smem;
}

// ---------------------------------------------------------------------------
// Coefficient transform on the tensor cores.
//
// For the points of a tile, the coefficient form A_a = sum_j M[j][a] c_j of
// every reference region is one dense product D = C M with C (points x union
// sites) and M (union sites x (region, monomial) columns) constant per spline.
// It runs as tcgen05.mma kind::tf32 with M = 128 rows (one point per TMEM
// lane, one thread per point), N = the column count rounded up to 16,
// K = the union sites rounded up to 8; FP32 accuracy from three TF32 products
// (split A = A_hi + A_lo, M = M_hi + M_lo: A_hi M_hi + A_hi M_lo + A_lo M_hi).
// C goes to tensor memory with tcgen05.st (each thread its own lane), M sits
// in shared memory in the K-major canonical layout without swizzle (8-row x
// 16-byte core matrices: K-adjacent ones 128 bytes apart, 8-row groups
// 8 * K * 4 bytes apart), D comes back with tcgen05.ld and feeds the same
// Horner forms as the FMA path.
// ---------------------------------------------------------------------------
struct TensorPlan {
    int nu = 0, kp = 0, ncol = 0, n = 0, cols = 0;
    std::vector<std::map<I3, std::vector<std::pair<int, double>>>> terms;
    std::vector<std::set<I3>> sup;
    std::vector<std::map<I3, int>> col;
};

// split: the coefficients need a TF32 hi + lo split (FP32 storage); BF16 and
// FP16 values are exact in TF32, so their A_lo rows and third product vanish.
// h16: the FP16 form (kind::f16, K steps of 16, two 16-bit values per column)
TensorPlan tensor_plan(const Table &t, const Stencil &st, bool split = true, bool h16 = false)
{
    TensorPlan p;
    const size_t K = t.ref.size();
    p.nu = (int)st.sites.size();
    p.kp = h16 ? (p.nu + 15) / 16 * 16 : (p.nu + 7) / 8 * 8;
    p.terms.resize(K);
    p.sup.resize(K);
    p.col.resize(K);
    for (size_t k = 0; k < K; ++k) {
        p.sup[k] = monomial_support(t.ref[k], st.region_to_union[k], p.terms[k]);
        for (const auto &m : p.sup[k]) p.col[k][m] = p.ncol++;
    }
    p.n = std::max(16, (p.ncol + 15) / 16 * 16);
    // one slot's columns: A hi, [A lo,] D (FP16: hi and lo take kp / 2 columns each)
    p.cols = ((h16 ? p.kp : (split ? 2 : 1) * p.kp) + p.n + 15) / 16 * 16;
    return p;
}

// round to the nearest FP16 value (ties to even; subnormals kept), as its bits
unsigned short fp16_bits(double v)
{
    if (v == 0.0) return std::signbit(v) ? 0x8000 : 0;
    const unsigned short sgn = v < 0 ? 0x8000 : 0;
    double a = std::fabs(v);
    if (a >= 65520.0) return sgn | 0x7c00;          // beyond the largest finite value: infinity
    int ex;
    std::frexp(a, &ex);                             // a = m 2^ex, 0.5 <= m < 1
    int e = ex - 1;                                 // a = 1.f 2^e
    if (e < -14) e = -14;                           // subnormal range: fixed step 2^-24
    const double q = std::nearbyint(std::ldexp(a, 10 - e));   // 11 significant bits (fewer below 2^-14)
    double r = std::ldexp(q, e - 10);
    // re-encode (the rounding may have carried into the next binade)
    int ex2;
    std::frexp(r, &ex2);
    int e2 = ex2 - 1;
    if (r >= 65520.0) return sgn | 0x7c00;
    if (e2 < -14) {                                 // subnormal: r = mant 2^-24
        return sgn | (unsigned short)std::lrint(std::ldexp(r, 24));
    }
    const unsigned short mant = (unsigned short)(std::lrint(std::ldexp(r, 10 - e2)) - 1024);
    return sgn | (unsigned short)((e2 + 15) << 10) | mant;
}

double fp16_value(unsigned short b)
{
    const int sgn = (b & 0x8000) ? -1 : 1, ex = (b >> 10) & 31, man = b & 1023;
    if (ex == 0) return sgn * std::ldexp((double)man, -24);
    return sgn * std::ldexp(1.0 + man / 1024.0, ex - 15);
}

// round to the nearest TF32 value (11 significant bits), ties away from zero
double tf32_round(double v)
{
    if (v == 0.0 || !std::isfinite(v)) return v;
    int ex;
    const double m = std::frexp(v, &ex);          // v = m 2^ex, 0.5 <= |m| < 1
    return std::ldexp(std::round(std::ldexp(m, 11)), ex - 11);
}

// power-of-two chunks of a register run for tcgen05.ld / st (x1 .. x64)
std::vector<std::pair<int, int>> pow2_chunks(int n)
{
    std::vector<std::pair<int, int>> r;
    int at = 0;
    for (int c = 64; c >= 1; c >>= 1)
        while (n - at >= c) {
            r.push_back({at, c});
            at += c;
        }
    return r;
}

}  // namespace

// The region-of-evaluation part of the classifier alone (the lines up to the
// site k0..k{D-1}), for kernels that first bound the sites of a block's points.
std::string roe_only(const Table &t)
{
    Emitter tmp;
    emit_classify(tmp, t);
    const std::string src = tmp.o.str();
    std::string keep;
    size_t pos = 0;
    int seen = 0;
    while (pos < src.size() && seen < t.dim) {
        const size_t nl = src.find('\n', pos);
        const std::string line = src.substr(pos, nl - pos + 1);
        keep += line;
        for (int q = 0; q < t.dim; ++q)
            if (line.find("const int k" + std::to_string(q) + " = ") != std::string::npos) ++seen;
        pos = nl + 1;
    }
    return keep;
}

// Slots (128-point tiles in flight) per block of the tensor-core kernel: as
// many as the 512 tensor-memory columns hold, at most 8 (1024 threads), at
// most 5 for the larger splines; var.tensor = 2..8 asks for fewer.
int tensor_slots(const Table &t, const ls_variant &var, ls_dtype dt)
{
    const TensorPlan p = tensor_plan(t, union_stencil(t), dt == LS_F32, dt == LS_F32 && var.tensor_kind == 1);
    // registers: a thread holds its next tile's K coefficients and its last
    // tile's N products; past 5 slots (640 threads, 102 registers each) the
    // larger splines spill (measured: BCC quintic BF16 at 6 slots)
    const int cap = (p.kp + p.n >= 64) ? 5 : 8;
    const int tmem_max = std::max(1, std::min(8, 512 / p.cols));
    int s = std::min(cap, tmem_max);
    // an explicit slot count (tensor >= 2) may go past the register cap, up to what tensor memory holds
    if (var.tensor >= 2) s = std::min(var.tensor, tmem_max);
    return s;
}

namespace {

// One block per SM (a block that allocates tensor memory is the only one on
// its SM) with S slots of 4 warps; each slot owns 128 points at a time, a
// column range of tensor memory, an mbarrier and an arrival counter (the
// last of its warps to stage a tile issues the product), and runs
// independently of the others.  Within a slot the tile loop is software
// pipelined: the gathers of tile t are issued before the results of tile
// t - 1 are read back, so the product of t - 1 runs behind them.
void emit_eval_kernel_tensor(Emitter &e, const Table &t, const ls_variant &var, const Stencil &st, int reach,
                             GenInfo &info, bool grad = false)
{
    const bool fold = t.fold == LS_FOLD_SIGNED_PERM;
    auto &o = e.o;
    const int D = t.dim;
    const size_t K = t.ref.size();
    const bool split = e.ld == "ls_ld_f32";     // BF16 / FP16 coefficients are exact in TF32
    // FP32 coefficients as FP16 products: each point's values scaled by a power
    // of two, split into FP16 hi (11 significant bits) + lo (the remainder),
    // three kind::f16 products, the row's scale undone on the results
    const bool h16 = split && var.tensor_kind == 1;
    const TensorPlan P = tensor_plan(t, st, split, h16);
    const int KP = P.kp, N = P.n, NU = P.nu, S = tensor_slots(t, var, split ? LS_F32 : LS_BF16);
    const int AC = h16 ? KP / 2 : KP;           // columns of one A split
    const int DC = split ? 2 * AC : AC;         // first accumulator column of a slot
    int alloc = 32;
    while (alloc < S * P.cols) alloc *= 2;
    info.tmem_cols = alloc;
    // the transform matrix (hi, then lo) in the canonical shared-memory order
    std::vector<double> B((size_t)N * KP, 0.0);
    for (size_t k = 0; k < K; ++k)
        for (const auto &m : P.sup[k])
            for (const auto &pr : P.terms[k].at(m)) B[(size_t)P.col[k].at(m) * KP + pr.first] += pr.second;
    // the table is emitted with the value kernel; the value + gradient kernel reads it too
    const std::string tab = "ls_tcB_" + kname(t, "eval");
    // FP16 form: the matrix scaled by 2^sB so that its largest entry lies in
    // [2^14, 2^15) (every entry and its lo part then far from the FP16 subnormals)
    int sB = 0;
    if (h16) {
        double bmax = 0.0;
        for (double v : B) bmax = std::max(bmax, std::fabs(v));
        int ex = 1;
        if (bmax > 0.0) std::frexp(bmax, &ex);      // bmax in [2^(ex-1), 2^ex)
        sB = 15 - ex;
    }
    if (!grad && h16) {
        // FP16 hi / lo bits, (n / 8) * 8 KP + (u / 8) * 64 + (n % 8) * 8 + (u % 8)
        o << "static __device__ const unsigned short " << tab << "[" << 2 * N * KP << "] = {\n";
        for (int h = 0; h < 2; ++h)
            for (int idx = 0; idx < N * KP; ++idx) {
                const int g = idx / (8 * KP), rem = idx % (8 * KP);
                const int ug = rem / 64, r2 = rem % 64;
                const int nn = g * 8 + r2 / 8, u = ug * 8 + r2 % 8;
                const double v = std::ldexp(B[(size_t)nn * KP + u], sB);
                const unsigned short hb = fp16_bits(v);
                const unsigned short bits = h == 0 ? hb : fp16_bits(v - fp16_value(hb));
                o << bits << ((idx + 1) % 16 == 0 ? ",\n" : ", ");
            }
        o << "};\n";
    }
    if (!grad && !h16) o << "static __device__ const float " << tab << "[" << 2 * N * KP << "] = {\n";
    for (int h = 0; h < (grad || h16 ? 0 : 2); ++h)
        for (int idx = 0; idx < N * KP; ++idx) {
            // idx = (n / 8) * 8 KP + (u / 4) * 32 + (n % 8) * 4 + (u % 4)
            const int g = idx / (8 * KP), rem = idx % (8 * KP);
            const int ug = rem / 32, r2 = rem % 32;
            const int nn = g * 8 + r2 / 4, u = ug * 4 + r2 % 4;
            const double v = B[(size_t)nn * KP + u];
            const double hi = tf32_round(v);
            o << flit(h == 0 ? hi : tf32_round(v - hi)) << ((idx + 1) % 8 == 0 ? ",\n" : ", ");
        }
    if (!grad && !h16) o << "};\n";
    // D FP32; A, B TF32 (2) or FP16 (0): always the same type for A and B
    const unsigned ab = h16 ? 0u : 2u;
    const unsigned idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((unsigned)(N >> 3) << 17) | ((128u >> 4) << 24);
    auto reglist = [](int cnt, int op0) {
        std::string r = "{";
        for (int q = 0; q < cnt; ++q) r += (q ? "," : "") + std::string("%") + std::to_string(op0 + q);
        return r + "}";
    };
    const int fma0 = e.fma;
    o << "extern \"C\" __global__ void __launch_bounds__(" << 128 * S << ", 1) "
      << kname(t, grad ? "eval_grad" : "eval") << "(const LsEvalArgs a)\n{\n";
    o << "  __shared__ __align__(1024) " << (h16 ? "unsigned short" : "float") << " ls_sB[" << 2 * N * KP << "];\n";
    o << "  __shared__ __align__(8) unsigned long long ls_bar[" << S << "];\n";
    o << "  __shared__ unsigned ls_cnt[" << S << "];\n";
    o << "  __shared__ unsigned ls_tbase;\n";
    o << "  const int E0 = a.e0, E1 = a.e1, E2 = a.e2, CS = a.cstride, CU = a.cunit;"
         " (void)E1; (void)E2; (void)CS; (void)CU;\n";
    o << "  const unsigned warp = threadIdx.x >> 5, slot = warp >> 2, lt = threadIdx.x & 127u;\n";
    o << "  for (int q = threadIdx.x; q < " << 2 * N * KP << "; q += blockDim.x) ls_sB[q] = " << tab << "[q];\n";
    o << "  if (warp == 0) {\n";
    o << "    asm volatile(\"tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\" :: "
         "\"r\"((unsigned)__cvta_generic_to_shared(&ls_tbase)), \"r\"(" << alloc << "u) : \"memory\");\n";
    o << "    asm volatile(\"tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\" ::: \"memory\");\n";
    o << "  }\n";
    o << "  if (threadIdx.x < " << S << ") {\n";
    o << "    asm volatile(\"mbarrier.init.shared::cta.b64 [%0], 1;\" :: "
         "\"r\"((unsigned)__cvta_generic_to_shared(&ls_bar[threadIdx.x])) : \"memory\");\n";
    o << "    ls_cnt[threadIdx.x] = 0u;\n";
    o << "  }\n";
    o << "  asm volatile(\"fence.proxy.async.shared::cta;\" ::: \"memory\");\n";
    o << "  asm volatile(\"tcgen05.fence::before_thread_sync;\" ::: \"memory\");\n";
    o << "  __syncthreads();\n";
    o << "  asm volatile(\"tcgen05.fence::after_thread_sync;\" ::: \"memory\");\n";
    o << "  const unsigned tm = ls_tbase + slot * " << P.cols << "u;      // this slot's columns\n";
    o << "  const unsigned tl = tm + ((32u * (warp & 3u)) << 16);   // and this warp's quarter of the lanes\n";
    o << "  const unsigned bar = (unsigned)__cvta_generic_to_shared(&ls_bar[slot]);\n";
    o << "  const unsigned lane = threadIdx.x & 31u;\n";
    o << "  const unsigned cnt = (unsigned)__cvta_generic_to_shared(&ls_cnt[slot]);   // warps staged, mod 4\n";
    o << "  const unsigned sb = (unsigned)__cvta_generic_to_shared(ls_sB);\n";
    o << "  unsigned phase = 0;\n  bool pending = false, bad = false;\n";
    o << "  long long pi = 0;\n  int pst = 2, ppsi = 0;\n  float pa0 = 0.0f, pa1 = 0.0f, pa2 = 0.0f;\n";
    if (h16) o << "  float pinv = 1.0f;   // the previous tile's scales (row and matrix), undone on its results\n";
    if (grad) {
        // the fold of the previous tile's point: reference axis and sign per Cartesian axis
        o << "  int pri0 = 0, pri1 = 1, pri2 = 2;\n  unsigned png0 = 0u, png1 = 0u, png2 = 0u;\n";
        o << "#define LS_OUT_OF_RANGE(V) { if (a.out) a.out[i] = (V);";
        for (int q = 0; q < D; ++q) o << " a.grad[(size_t)i * " << D << " + " << q << "] = (V);";
        o << " }\n";
    } else {
        o << "#define LS_OUT_OF_RANGE(V) { a.out[i] = (V); }\n";
    }
    o << "  for (long long tile = (long long)blockIdx.x * " << S << " + slot; ; tile += (long long)gridDim.x * " << S
      << ") {\n";
    // chunked: past 5 slots a large spline reads the products back in 8-column
    // pieces, each just before the polynomial's first use of it, so that the
    // next tile's gathered values and all of the products are not live
    // together (72-80 registers instead of 96 and more: 6 slots fit without
    // spilling)
    const bool chunked = S > 5 && P.kp + P.n >= 64;
    o << "    const bool have = tile * 128 < a.n;\n";
    o << "    const long long i = tile * 128 + lt;\n";
    o << "    int stt = 2;\n";
    for (int q = 0; q < 3; ++q) o << "    float x" << q << " = 0.0f;\n";
    o << "    if (have && i < a.n) {\n";
    for (int q = 0; q < D; ++q) o << "      x" << q << " = ls_ld_pt(a.pts + (size_t)i * " << D << " + " << q << ");\n";
    o << "      if (";
    for (int q = 0; q < D; ++q) o << (q ? " && " : "") << "fabsf(x" << q << ") < 4194304.0f";
    o << ") stt = 0;\n      else {\n        const bool isn = ";
    for (int q = 0; q < D; ++q) o << (q ? " || " : "") << "(x" << q << " != x" << q << ")";
    o << ";\n        LS_OUT_OF_RANGE(isn ? __int_as_float(0x7fffffff) : 0.0f);\n        stt = 1;\n      }\n    }\n";
    for (int j = 0; j < KP; ++j) o << "    float tc" << j << " = 0.0f;\n";
    o << "    float ta0 = 0.0f, ta1 = 0.0f, ta2 = 0.0f;\n    int tpsi = 0;\n";
    if (grad) o << "    int tri0 = 0, tri1 = 1, tri2 = 2;\n    unsigned tng0 = 0u, tng1 = 0u, tng2 = 0u;\n";
    o << "    if (stt == 0) {\n";
    emit_classify(e, t);
    emit_gathers(e, t, st.sites, reach, "a.coef", false, true, var.group, var.depth);
    for (int j = 0; j < NU; ++j) o << "    tc" << j << " = c" << j << ";\n";
    for (int q = 0; q < D; ++q) o << "    ta" << q << " = a" << q << ";\n";
    o << "    tpsi = psi;\n";
    if (grad && fold)
        for (int q = 0; q < D; ++q) o << "    tri" << q << " = ri" << q << "; tng" << q << " = ng" << q << ";\n";
    o << "    }\n";
    // results of the previous tile
    o << "    if (pending) {\n";
    // each warp waits for the product on its own (lane 0 polls)
    o << "      unsigned okw = 1u;\n";
    o << "      if (lane == 0) okw = ls_mbar_poll(bar, phase, a.status) ? 1u : 0u;\n";
    o << "      okw = __shfl_sync(0xffffffffu, okw, 0);\n";
    o << "      if (!okw) { bad = true; break; }\n";
    o << "      phase ^= 1u;\n";
    o << "      asm volatile(\"tcgen05.fence::after_thread_sync;\" ::: \"memory\");\n";
    for (int q = 0; q < N; ++q) o << "      unsigned td" << q << ";\n";
    auto emit_ld = [&](std::ostream &os, int first, int cnt) {
        os << "      asm volatile(\"tcgen05.ld.sync.aligned.32x32b.x" << cnt << ".b32 " << reglist(cnt, 0) << ", [%"
           << cnt << "];\" : ";
        for (int q = 0; q < cnt; ++q) os << (q ? ", " : "") << "\"=r\"(td" << (first + q) << ")";
        os << " : \"r\"(tl + " << (DC + first) << "u) : \"memory\");\n";
    };
    std::vector<std::vector<std::string>> fk;
    if (!chunked) {
        for (const auto &ch : pow2_chunks(N)) emit_ld(o, ch.first, ch.second);
        o << "      asm volatile(\"tcgen05.wait::ld.sync.aligned;\" ::: \"memory\");\n";
        o << "      if (pst == 0) {\n";
        for (int q = 0; q < D; ++q) o << "      const float a" << q << " = pa" << q << ";\n";
        o << "      const int psi = ppsi; (void)psi;\n";
        for (size_t k = 0; k < K; ++k) {
            std::map<I3, std::string> pre;
            for (const auto &m : P.sup[k]) {
                const std::string nm = "tA" + std::to_string(P.col[k].at(m));
                o << "      const float " << nm << " = __uint_as_float(td" << P.col[k].at(m) << ")"
                  << ";\n";
                pre[m] = nm;
            }
            fk.push_back(emit_region_poly(e, t, (int)k, st.region_to_union[k], grad ? 1 : 0, &pre));
        }
    } else {
        // the polynomials for every lane (the loads are warp-collective), each
        // 8-column piece loaded right before the first line that reads it
        for (int q = 0; q < D; ++q) o << "      const float a" << q << " = pa" << q << ";\n";
        o << "      const int psi = ppsi; (void)psi;\n";
        const std::string before = o.str();
        o.str("");
        for (size_t k = 0; k < K; ++k) {
            std::map<I3, std::string> pre;
            for (const auto &m : P.sup[k]) pre[m] = "__uint_as_float(td" + std::to_string(P.col[k].at(m)) + ")";
            fk.push_back(emit_region_poly(e, t, (int)k, st.region_to_union[k], grad ? 1 : 0, &pre));
        }
        const std::string poly = o.str();
        o.str("");
        o << before;
        std::vector<bool> loaded(N / 8, false);
        size_t pos = 0;
        while (pos < poly.size()) {
            size_t end = poly.find('\n', pos);
            if (end == std::string::npos) end = poly.size() - 1;
            const std::string line = poly.substr(pos, end - pos + 1);
            bool any = false;
            for (size_t f = line.find("(td"); f != std::string::npos; f = line.find("(td", f + 3)) {
                size_t d = f + 3;
                int col = 0;
                while (d < line.size() && std::isdigit((unsigned char)line[d])) col = col * 10 + (line[d++] - '0');
                if (d > f + 3 && !loaded[col / 8]) {
                    emit_ld(o, col / 8 * 8, 8);
                    loaded[col / 8] = true;
                    any = true;
                }
            }
            if (any) o << "      asm volatile(\"tcgen05.wait::ld.sync.aligned;\" ::: \"memory\");\n";
            o << line;
            pos = end + 1;
        }
        o << "      if (pst == 0) {\n";
    }
    // value and (reference-frame) gradient, the region picked by psi
    std::vector<std::string> out;
    for (int c = 0; c < (grad ? D + 1 : 1); ++c) {
        std::string sel = fk[K - 1][c];
        for (int k = (int)K - 2; k >= 0; --k)
            sel = "(psi == " + std::to_string(k) + ") ? " + fk[k][c] + " : (" + sel + ")";
        const std::string nm = c == 0 ? "tf" : "tg" + std::to_string(c - 1);
        // FP16 form: the results are linear in the products, so both scales come off once here
        o << "      const float " << nm << " = " << (h16 ? "pinv * (" + sel + ")" : sel) << ";\n";
        out.push_back(nm);
    }
    if (!grad) {
        o << "      ls_st_out(a.out + pi, tf);\n";
    } else {
        o << "      if (a.out) ls_st_out(a.out + pi, tf);\n";
        // back to Cartesian axes: df/dx_i = sign_i * g[reference axis landing on i]
        for (int q = 0; q < D; ++q) {
            if (fold) {
                o << "      { const float gg = ";
                for (int r = 0; r < D - 1; ++r) o << "(pri" << q << " == " << r << ") ? " << out[1 + r] << " : ";
                o << out[D] << "; a.grad[(size_t)pi * " << D << " + " << q << "] = png" << q << " ? -gg : gg; }\n";
            } else {
                o << "      a.grad[(size_t)pi * " << D << " + " << q << "] = " << out[1 + q] << ";\n";
            }
        }
    }
    o << "      }\n";
    o << "      pending = false;\n";
    o << "    }\n";
    o << "    if (!have) break;\n";
    // split and stage this tile's coefficients (slot columns [0, KP) hi, [KP, 2 KP) lo).
    // With several reference regions the gathers cover their union: the sites
    // outside the point's own region are zeroed first (their weights vanish
    // there), so that neither the row scale nor a non-finite value of a site
    // the point does not use reaches its products (0 x inf would be NaN).
    if (K > 1) {
        for (int u = 0; u < NU; ++u) {
            std::vector<int> regs;
            for (size_t k = 0; k < K; ++k)
                if (std::find(st.region_to_union[k].begin(), st.region_to_union[k].end(), u) !=
                    st.region_to_union[k].end())
                    regs.push_back((int)k);
            if (regs.size() == K) continue;
            o << "    if (";
            for (size_t r = 0; r < regs.size(); ++r) o << (r ? " && " : "") << "tpsi != " << regs[r];
            if (regs.empty()) o << "true";
            o << ") tc" << u << " = 0.0f;\n";
        }
    }
    if (h16) {
        // the row's scale: a power of two that brings max |c_j| into [2^14, 2^15)
        // (biased exponent teb: tsc = 2^(141 - teb); rows below 2^-112 keep less scaling)
        o << "    float tmx = 0.0f;\n";
        for (int j = 0; j < KP; ++j) o << "    tmx = fmaxf(tmx, fabsf(tc" << j << "));\n";
        o << "    const int teb = min(max((int)(__float_as_uint(tmx) >> 23), 15), 252);\n";
        o << "    const float tsc = __uint_as_float((unsigned)(268 - teb) << 23);\n";
        o << "    const float tinv = __uint_as_float((unsigned)(teb - 14) << 23) * " << flit(std::ldexp(1.0, -sB))
          << ";\n";
        // hi: the scaled value with its low 13 mantissa bits cleared (11
        // significant bits, an FP16 value wherever FP16 is normal); lo: the exact
        // remainder, rounded to FP16.  Two values per 32-bit column, the even K
        // index in the low half (cvt.rn.f16x2.f32 puts its first operand high).
        for (int q = 0; q < KP / 2; ++q) {
            o << "    unsigned th" << q << ", tw" << q << ";\n";
            o << "    { const float v0 = tc" << 2 * q << " * tsc, v1 = tc" << 2 * q + 1 << " * tsc;\n";
            o << "      const float h0 = __uint_as_float(__float_as_uint(v0) & 0xffffe000u);\n";
            o << "      const float h1 = __uint_as_float(__float_as_uint(v1) & 0xffffe000u);\n";
            o << "      asm(\"cvt.rn.f16x2.f32 %0, %1, %2;\" : \"=r\"(th" << q << ") : \"f\"(h1), \"f\"(h0));\n";
            o << "      asm(\"cvt.rn.f16x2.f32 %0, %1, %2;\" : \"=r\"(tw" << q << ") : \"f\"(v1 - h1), \"f\"(v0 - h0)); }\n";
        }
    }
    for (int j = 0; j < (h16 ? 0 : KP); ++j) {
        if (split) {
            o << "    unsigned th" << j << ", tw" << j << ";\n";
            o << "    asm(\"cvt.rna.tf32.f32 %0, %1;\" : \"=r\"(th" << j << ") : \"f\"(tc" << j << "));\n";
            o << "    tw" << j << " = __float_as_uint(tc" << j << " - __uint_as_float(th" << j << "));\n";
        } else {
            o << "    const unsigned th" << j << " = __float_as_uint(tc" << j << ");   // exact in TF32\n";
        }
    }
    for (int h = 0; h < (split ? 2 : 1); ++h)
        for (const auto &ch : pow2_chunks(AC)) {
            o << "    asm volatile(\"tcgen05.st.sync.aligned.32x32b.x" << ch.second << ".b32 [%0], "
              << reglist(ch.second, 1) << ";\" :: \"r\"(tl + " << (h * AC + ch.first) << "u)";
            for (int q = 0; q < ch.second; ++q) o << ", \"r\"(" << (h ? "tw" : "th") << (ch.first + q) << ")";
            o << " : \"memory\");\n";
        }
    o << "    asm volatile(\"tcgen05.wait::st.sync.aligned;\" ::: \"memory\");\n";
    o << "    asm volatile(\"tcgen05.fence::before_thread_sync;\" ::: \"memory\");\n";
    // no barrier: each warp counts itself in (release / acquire on the slot's
    // counter); the fourth warp of the tile issues the product, which thereby
    // follows every warp's tcgen05.st of this tile and tcgen05.ld of the last
    o << "    __syncwarp();\n";
    o << "    unsigned arrived = 0u;\n";
    o << "    if (lane == 0) asm volatile(\"atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;\" : \"=r\"(arrived) : "
         "\"r\"(cnt) : \"memory\");\n";
    o << "    if (lane == 0 && (arrived & 3u) == 3u) {\n";
    o << "      asm volatile(\"tcgen05.fence::after_thread_sync;\" ::: \"memory\");\n";
    // smem descriptors: start >> 4, LBO 128 B, SBO = 8 rows of K elements, version 1, no swizzle
    const int eb = h16 ? 2 : 4;                 // bytes per element
    o << "      const unsigned long long dbase = ((unsigned long long)(" << 8 * KP * eb << " >> 4) << 32) |"
         " ((unsigned long long)(128 >> 4) << 16) | (1ull << 46);\n";
    const std::string mma = std::string("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::") +
                            (h16 ? "f16" : "tf32") + " [%0], [%1], %2, %3, p; }";
    struct Prod { int acol; int boff; };
    const Prod prods[3] = {{0, 0}, {0, N * KP * eb}, {AC, 0}};
    const int kstep = h16 ? 16 : 8;              // K elements per product instruction (32 bytes)
    for (int pi = 0; pi < (split ? 3 : 2); ++pi)
        for (int s2 = 0; s2 < KP / kstep; ++s2) {
            o << "      asm volatile(\"" << mma << "\" :: \"r\"(tm + " << DC << "u), \"r\"(tm + "
              << (prods[pi].acol + 8 * s2) << "u), \"l\"(dbase | (unsigned long long)(((sb + "
              << (prods[pi].boff + 256 * s2) << "u) & 0x3FFFFu) >> 4)), \"r\"(" << idesc << "u), \"r\"("
              << ((pi == 0 && s2 == 0) ? 0 : 1) << "u) : \"memory\");\n";
        }
    o << "      asm volatile(\"tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\" :: "
         "\"r\"(bar) : \"memory\");\n";
    o << "    }\n";
    o << "    pending = true;\n    pi = i;\n    pst = stt;\n    ppsi = tpsi;\n";
    if (h16) o << "    pinv = tinv;\n";
    for (int q = 0; q < D; ++q) o << "    pa" << q << " = ta" << q << ";\n";
    if (grad)
        for (int q = 0; q < D; ++q) o << "    pri" << q << " = tri" << q << "; png" << q << " = tng" << q << ";\n";
    o << "  }\n#undef LS_OUT_OF_RANGE\n";
    // a wait that gave up: wait once more (bounded) for the products in flight
    // before the tensor memory is released
    o << "  if (bad && lane == 0) ls_mbar_poll(bar, phase, 0);\n";
    o << "  asm volatile(\"tcgen05.fence::before_thread_sync;\" ::: \"memory\");\n";
    o << "  __syncthreads();\n";
    o << "  if (warp == 0) asm volatile(\"tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\" :: \"r\"(ls_tbase), \"r\"("
      << alloc << "u) : \"memory\");\n";
    o << "}\n\n";
    if (grad) info.fma_grad = e.fma - fma0;
    else info.fma_value = e.fma - fma0;
}

// Tile edge (grid indices per axis) of the staged kernel: var.stage when > 1,
// else 12 for the scale-2 lattices and 16 for the Cartesian one.
int stage_edge(const Table &t, const ls_variant &var)
{
    if (var.stage > 1) return var.stage;
    return t.scale == 2 ? 12 : 16;
}

// Tile-staged value kernel for spatially sorted points.  A block takes a tile
// of blockDim consecutive points, reduces the bounding box of their
// region-of-evaluation sites, and if that box plus the stencil reach fits the
// fixed shared-memory tile, one thread loads the coefficient box with a single
// TMA tensor copy (cp.async.bulk.tensor; out-of-bounds elements arrive as 0,
// which is the zero extension beyond the arrays) completing on an mbarrier.
// Every point of the tile is then evaluated by the same point code reading the
// tile (coordinates shifted by an even integer vector, so y, the fold and the
// arithmetic are unchanged); tiles that do not fit, and non-finite or far
// points, take the global path.  a.tmap: the volume's tensor map (NULL: always
// the global path).  The wait is bounded: on timeout *a.status is set and the
// block leaves.  Returns the tile's dynamic shared memory in bytes.
int emit_eval_kernel_staged(Emitter &e, const Table &t, const ls_variant &var, const Stencil &st, int reach,
                            GenInfo &info)
{
    auto &o = e.o;
    const int D = t.dim;
    const int C = (int)t.cosets.size();
    const int sc = t.scale;
    // tile edge in grid indices per axis (per coset): var.stage > 1 sets it
    const int edge = stage_edge(t, var);
    const int BQ[3] = {edge, edge, edge};
    info.stage_edge = edge;
    // the copy's x start must be a multiple of 16 bytes: qlo0 * C floats in the
    // interleaved map, qlo0 floats in the coset-major one
    const int align_inter = (C >= 4) ? 1 : 4 / C;
    const int tile_floats = BQ[0] * BQ[1] * BQ[2] * C;
    const int fma0 = e.fma;
    const std::string pf_g = kname(t, "eval_pt");
    const std::string pf_s = kname(t, "eval_pt_tile");
    emit_eval_point(e, t, var, st, reach, false, pf_g);
    const std::string ld_save = e.ld;
    e.ld = "ls_sh_ld";
    emit_eval_point(e, t, var, st, reach, false, pf_s, true);
    e.ld = ld_save;
    info.fma_value = (e.fma - fma0) / 2;
    o << "extern \"C\" __global__ void __launch_bounds__(" << var.block;
    if (var.min_blocks > 0) o << ", " << var.min_blocks;
    o << ") " << kname(t, "eval") << "(const LsEvalArgs a)\n{\n";
    // the tensor copy's destination: the dynamic buffer rounded up to 128 bytes
    // (the buffer is allocated 128 bytes longer than the tile)
    o << "  extern __shared__ __align__(128) float ls_dyn[];\n";
    o << "  __shared__ __align__(8) unsigned long long ls_bar;\n";
    o << "  __shared__ int s_lo[3], s_hi[3];\n";
    o << "  const unsigned bar = (unsigned)__cvta_generic_to_shared(&ls_bar);\n";
    o << "  const unsigned dyn = (unsigned)__cvta_generic_to_shared(ls_dyn);\n";
    o << "  const unsigned dst = (dyn + 127u) & ~127u;\n";
    o << "  float* const ls_tile = ls_dyn + (dst - dyn) / 4u;\n";
    o << "  if (threadIdx.x == 0) asm volatile(\"mbarrier.init.shared::cta.b64 [%0], 1;\" :: \"r\"(bar) : \"memory\");\n";
    o << "  unsigned phase = 0;\n";
    o << "  const long long B = blockDim.x;\n";
    o << "  for (long long t0 = (long long)blockIdx.x * B; t0 < a.n; t0 += (long long)gridDim.x * B) {\n";
    o << "    if (threadIdx.x < 3) { s_lo[threadIdx.x] = 0x7fffffff; s_hi[threadIdx.x] = -0x7fffffff; }\n";
    o << "    __syncthreads();\n";
    o << "    const long long i = t0 + threadIdx.x;\n";
    o << "    float x0 = 0.0f, x1 = 0.0f, x2 = 0.0f;\n";
    o << "    bool good = false;\n";
    o << "    int kk[3] = {0, 0, 0};\n";
    o << "    if (i < a.n) {\n";
    o << "      x0 = ls_ld_pt(a.pts + (size_t)i * " << D << ");\n";
    o << "      x1 = ls_ld_pt(a.pts + (size_t)i * " << D << " + 1);\n";
    if (D == 3) o << "      x2 = ls_ld_pt(a.pts + (size_t)i * 3 + 2);\n";
    o << "      good = fabsf(x0) < 4194304.0f && fabsf(x1) < 4194304.0f && fabsf(x2) < 4194304.0f;\n";
    o << "    }\n";
    o << "    if (good) {\n";
    // region-of-evaluation site (the same decoding as the point code)
    o << roe_only(t);
    for (int q = 0; q < D; ++q) o << "      kk[" << q << "] = k" << q << ";\n";
    o << "    }\n";
    // block bounding box of the sites
    o << "    {\n";
    for (int q = 0; q < D; ++q) {
        o << "      int lo" << q << " = good ? kk[" << q << "] : 0x7fffffff, hi" << q << " = good ? kk[" << q
          << "] : -0x7fffffff;\n";
        o << "      lo" << q << " = __reduce_min_sync(0xffffffffu, lo" << q << "); hi" << q
          << " = __reduce_max_sync(0xffffffffu, hi" << q << ");\n";
        o << "      if ((threadIdx.x & 31) == 0) { atomicMin(&s_lo[" << q << "], lo" << q << "); atomicMax(&s_hi[" << q
          << "], hi" << q << "); }\n";
    }
    o << "    }\n";
    o << "    __syncthreads();\n";
    // tile origin in grid indices and whether the stencils fit
    o << "    int qlo[3] = {0, 0, 0};\n    bool fits = a.tmap != 0 && s_lo[0] <= s_hi[0];\n";
    o << "    const int al = " << (C == 1 ? std::string("4") : "(a.cstride == 1) ? " + std::to_string(align_inter) + " : 4")
      << ";\n";
    for (int q = 0; q < D; ++q) {
        if (sc == 2) {
            o << "    qlo[" << q << "] = (s_lo[" << q << "] - " << reach << ") >> 1;\n";
            if (q == 0) o << "    qlo[0] &= ~(al - 1);\n";
            o << "    fits = fits && ((s_hi[" << q << "] + " << reach << ") >> 1) - qlo[" << q << "] < " << BQ[q] << ";\n";
        } else {
            o << "    qlo[" << q << "] = s_lo[" << q << "] - " << reach << ";\n";
            if (q == 0) o << "    qlo[0] &= ~(al - 1);\n";
            o << "    fits = fits && (s_hi[" << q << "] + " << reach << ") - qlo[" << q << "] < " << BQ[q] << ";\n";
        }
    }
    // qlo >= 0: x - scale * qlo is then exact in FP32 (a multiple of ulp(x),
    // no larger than x), so the tile path computes bit-identical results
    o << "    fits = fits && qlo[0] >= 0 && qlo[1] >= 0 && qlo[2] >= 0;\n";
    o << "    if (fits) {\n";
    o << "      if (threadIdx.x == 0) {\n";
    o << "        asm volatile(\"fence.proxy.async.shared::cta;\" ::: \"memory\");\n";
    o << "        asm volatile(\"mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\" :: \"r\"(bar), \"r\"("
      << tile_floats * 4 << ") : \"memory\");\n";
    // coordinates: interleaved layout (3D map: (E0*C, E1, E2)) or coset-major (4D map: (E0, E1, E2, C))
    o << "        if (" << (C == 1 ? "true" : "a.cstride == 1") << ") {\n";
    o << "          asm volatile(\"cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
         " [%0], [%1, {%2, %3, %4}], [%5];\" :: \"r\"(dst), \"l\"(a.tmap), \"r\"(qlo[0] * " << C
      << "), \"r\"(qlo[1]), \"r\"(qlo[2]), \"r\"(bar) : \"memory\");\n";
    o << "        } else {\n";
    o << "          asm volatile(\"cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
         " [%0], [%1, {%2, %3, %4, %5}], [%6];\" :: \"r\"(dst), \"l\"(a.tmap), \"r\"(qlo[0]), \"r\"(qlo[1]),"
         " \"r\"(qlo[2]), \"r\"(0), \"r\"(bar) : \"memory\");\n";
    o << "        }\n      }\n";
    o << "      const bool ok = ls_mbar_wait(bar, phase, a.status);\n";
    o << "      if (__syncthreads_or(!ok)) return;\n";
    o << "      phase ^= 1u;\n";
    o << "      if (good) {\n";
    o << "        LsEvalArgs b = a;\n";
    o << "        b.coef = ls_tile; b.e0 = " << BQ[0] << "; b.e1 = " << BQ[1] << "; b.e2 = " << (D == 3 ? BQ[2] : 1)
      << ";\n";
    o << "        if (" << (C == 1 ? "true" : "a.cstride == 1") << ") { b.cstride = 1; b.cunit = " << C
      << "; } else { b.cstride = "
      << BQ[0] * BQ[1] * BQ[2] << "; b.cunit = 1; }\n";
    o << "        " << pf_s << "(b, i, x0 - " << sc << ".0f * (float)qlo[0], x1 - " << sc << ".0f * (float)qlo[1], "
      << (D == 3 ? "x2 - " + std::to_string(sc) + ".0f * (float)qlo[2]" : std::string("0.0f")) << ");\n";
    o << "      } else if (i < a.n) {\n";
    o << "        " << pf_g << "(a, i);\n";
    o << "      }\n";
    o << "    } else if (i < a.n) {\n";
    o << "      " << pf_g << "(a, i);\n";
    o << "    }\n";
    o << "    __syncthreads();\n";
    o << "  }\n}\n\n";
    return tile_floats * 4 + 128;
}

// Per-site weight polynomials w_j(u) (weights form), for the adjoint.
// Returns the name of w for union site j (or "" if identically 0 in all regions).
std::vector<std::string> emit_site_weights(Emitter &e, const Table &t, const Stencil &st)
{
    auto &o = e.o;
    const int D = t.dim;
    const size_t K = t.ref.size();
    std::vector<std::vector<std::string>> per(K, std::vector<std::string>(st.sites.size()));
    for (size_t k = 0; k < K; ++k) {
        const RefRegion &r = t.ref[k];
        std::string uv[3];
        for (int i = 0; i < D; ++i) {
            uv[i] = "u" + std::to_string(k) + "_" + std::to_string(i);
            o << "    const float " << uv[i] << " = a" << i << " - " << flit(r.center[i]) << ";\n";
        }
        const size_t nm = r.mono.size();
        for (size_t j = 0; j < r.sites.size(); ++j) {
            std::map<I3, std::vector<std::pair<int, double>>> terms;
            std::set<I3> sup;
            for (size_t aa = 0; aa < nm; ++aa) {
                double c = r.coef[j * nm + aa];
                if (c == 0.0) continue;
                sup.insert(r.mono[aa]);
                terms[r.mono[aa]].push_back({0, c});
            }
            PolyEmit pe{e, D, "", {uv[0], uv[1], uv[2]}, {}, {}};
            auto coefc = [&](const I3 &m) -> std::string {
                auto it = terms.find(m);
                return it == terms.end() ? std::string() : flit(it->second[0].second);
            };
            std::string w = pe.horner(0, I3{0, 0, 0}, coefc, sup);
            if (w.empty()) continue;
            std::string nmv = e.fresh("w");
            o << "    const float " << nmv << " = " << w << ";\n";
            per[k][st.region_to_union[k][j]] = nmv;
        }
    }
    std::vector<std::string> out(st.sites.size());
    for (size_t j = 0; j < st.sites.size(); ++j) {
        if (K == 1) {
            out[j] = per[0][j];
            continue;
        }
        bool any = false;
        for (size_t k = 0; k < K; ++k) any = any || !per[k][j].empty();
        if (!any) continue;
        std::string sel = per[K - 1][j].empty() ? "0.0f" : per[K - 1][j];
        for (int k = (int)K - 2; k >= 0; --k)
            sel = "(psi == " + std::to_string(k) + ") ? " + (per[k][j].empty() ? "0.0f" : per[k][j]) + " : (" + sel + ")";
        std::string nmv = e.fresh("ws");
        o << "    const float " << nmv << " = " << sel << ";\n";
        out[j] = nmv;
    }
    return out;
}

// Atomic adjoint: dcoef[site] += g * w_site for every stencil site of every point.
// Scatter-add flavours of the point-wise adjoint.
// The adjoint's work for one point whose coordinates x0.. and gout value gp
// are loaded: classify (kshift: sites relative to an integer origin), the
// site weights, the site addresses (ad_j, -1 beyond the arrays) and one add
// per site, add(address variable, value expression) giving the statement.
void emit_adjoint_body(Emitter &e, const Table &t, const Stencil &st, int reach,
                       const std::function<std::string(const std::string &, const std::string &)> &add,
                       const char *kshift = nullptr)
{
    auto &o = e.o;
    const int D = t.dim;
    emit_classify(e, t, kshift);
    if (!t.sep.empty()) {
        // weights per axis
        for (int i = 0; i < D; ++i) {
            const Axis &ax = t.sep[i];
            o << "    const float su" << i << " = y" << i << " - " << flit(ax.center) << ";\n";
            const int nc = ax.degree + 1;
            for (size_t j = 0; j < ax.sites.size(); ++j) {
                std::string acc = flit(ax.coef[j * nc + ax.degree]);
                for (int d = ax.degree - 1; d >= 0; --d)
                    acc = "fmaf(" + acc + ", su" + std::to_string(i) + ", " + flit(ax.coef[j * nc + d]) + ")";
                o << "    const float w" << i << "_" << j << " = " << acc << ";\n";
            }
        }
        const int n0 = (int)t.sep[0].sites.size(), n1 = D > 1 ? (int)t.sep[1].sites.size() : 1,
                  n2 = D > 2 ? (int)t.sep[2].sites.size() : 1;
        std::vector<I3> sites;
        for (int j2 = 0; j2 < n2; ++j2)
            for (int j1 = 0; j1 < n1; ++j1)
                for (int j0 = 0; j0 < n0; ++j0)
                    sites.push_back({t.sep[0].sites[j0], D > 1 ? t.sep[1].sites[j1] : 0, D > 2 ? t.sep[2].sites[j2] : 0});
        int rch = 0;
        for (auto &s : sites)
            for (int i = 0; i < D; ++i) rch = std::max(rch, std::abs(s[i]));
        emit_gathers(e, t, sites, rch, "", true, false);
        for (int j2 = 0; j2 < n2; ++j2)
            for (int j1 = 0; j1 < n1; ++j1) {
                o << "    { const float gw = gp * w1_" << j1 << (D > 2 ? " * w2_" + std::to_string(j2) : std::string()) << ";\n";
                for (int j0 = 0; j0 < n0; ++j0) {
                    int j = (j2 * n1 + j1) * n0 + j0;
                    o << "      " << add("ad" + std::to_string(j), "gw * w0_" + std::to_string(j0)) << "\n";
                }
                o << "    }\n";
            }
    } else {
        auto w = emit_site_weights(e, t, st);
        emit_gathers(e, t, st.sites, reach, "", true, false);
        for (size_t j = 0; j < st.sites.size(); ++j) {
            if (w[j].empty()) continue;
            o << "    " << add("ad" + std::to_string(j), "gp * " + w[j]) << "\n";
        }
    }
}

enum AdjFlavour { ADJ_ATOMIC, ADJ_WARPAGG, ADJ_FIXED };

void emit_adjoint_atomic(Emitter &e, const Table &t, const ls_variant &var, const Stencil &st, int reach,
                         AdjFlavour fl)
{
    auto &o = e.o;
    // one scatter-add of value V at address variable AD
    auto add = [&](const std::string &ad, const std::string &v) {
        if (fl == ADJ_WARPAGG) return "ls_agg_add(a.dcoef, " + ad + ", " + v + ");";
        if (fl == ADJ_FIXED)
            return "if (" + ad + " >= 0) atomicAdd(a.iacc + " + ad + ", (unsigned long long)__float2ll_rn((" + v +
                   ") * isc));";
        return "if (" + ad + " >= 0) atomicAdd(a.dcoef + " + ad + ", " + v + ");";
    };
    const char *what = fl == ADJ_WARPAGG ? "adjoint_warpagg" : fl == ADJ_FIXED ? "adjoint_fixed" : "adjoint_atomic";
    o << "extern \"C\" __global__ void __launch_bounds__(" << var.block << ") " << kname(t, what)
      << "(const LsAdjArgs a)\n{\n";
    // fixed point: each value is rounded to an integer multiple of 2^-s and summed
    // exactly in int64, so the result does not depend on the order of the atomics
    if (fl == ADJ_FIXED) o << "  const float isc = __ldg(a.iscale);\n";
    o << "  const int E0 = a.e0, E1 = a.e1, E2 = a.e2, CS = a.cstride, CU = a.cunit;"
         " (void)E1; (void)E2; (void)CS; (void)CU;\n";
    o << "  const long long stride = (long long)gridDim.x * blockDim.x;\n";
    o << "#define LS_OUT_OF_RANGE(V) { }\n";
    o << "  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {\n";
    emit_point_load(e, t);
    o << "    const float gp = __ldg(a.gout + i);\n";
    o << "    if (gp == 0.0f) continue;\n";
    emit_adjoint_body(e, t, st, reach, add);
    o << "  }\n#undef LS_OUT_OF_RANGE\n}\n\n";
}


// Tile edge (grid indices per axis) of the tiled adjoint: var.stage when > 1,
// else the largest edge up to 16 (scale 2) or 24 (Cartesian) whose tile of
// elem-byte values per coset takes at most 48 KiB of shared memory.
int adjoint_tile_edge(const Table &t, const ls_variant &var, int elem)
{
    if (var.stage > 1) return var.stage;
    const int C = (int)t.cosets.size();
    int edge = t.scale == 2 ? 16 : 24;
    auto bytes = [&](int e) {
        long long v = (long long)C * elem;
        for (int q = 0; q < t.dim; ++q) v *= e;
        return v;
    };
    while (edge > 4 && bytes(edge) > 48 * 1024) --edge;
    return edge;
}

// Tiled adjoint for spatially sorted points.  A block takes blockDim
// consecutive points, bounds their region-of-evaluation sites, and if their
// stencils fit one tile of TE^D grid indices per coset, accumulates the
// points' contributions in shared memory (the tile as a small interleaved
// volume: element q * C + j) and then adds every nonzero tile element to
// global memory once: one global atomic per touched coefficient instead of
// one per (point, site).  Other blocks take the per-point path.  fixed: the
// values are the fixed-point integers of the deterministic mode, summed with
// 64-bit integer atomics in shared and global memory (the same integers as
// the untiled fixed-point kernel, so the same bits).  Returns the dynamic
// shared memory in bytes.
int emit_adjoint_tiled(Emitter &e, const Table &t, const ls_variant &var, const Stencil &st, int reach, bool fixed)
{
    auto &o = e.o;
    const int D = t.dim;
    const int C = (int)t.cosets.size();
    const int sc = t.scale;
    const int TE = adjoint_tile_edge(t, var, fixed ? 8 : 4);
    int TN = C;
    for (int q = 0; q < D; ++q) TN *= TE;
    const char *T = fixed ? "unsigned long long" : "float";
    auto gadd = [&](const std::string &ad, const std::string &v) -> std::string {
        if (fixed)
            return "if (" + ad + " >= 0) atomicAdd(a.iacc + " + ad + ", (unsigned long long)__float2ll_rn((" + v +
                   ") * isc));";
        return "if (" + ad + " >= 0) atomicAdd(a.dcoef + " + ad + ", " + v + ");";
    };
    auto tadd = [&](const std::string &ad, const std::string &v) -> std::string {
        if (fixed)
            return "if (" + ad + " >= 0) atomicAdd(ls_tile + " + ad + ", (unsigned long long)__float2ll_rn((" + v +
                   ") * isc));";
        return "if (" + ad + " >= 0) atomicAdd(ls_tile + " + ad + ", " + v + ");";
    };
    o << "extern \"C\" __global__ void __launch_bounds__(" << var.block << ") "
      << kname(t, fixed ? "adjoint_tile_fixed" : "adjoint_tile") << "(const LsAdjArgs a)\n{\n";
    o << "  extern __shared__ __align__(16) unsigned char ls_tsm[];\n";
    o << "  " << T << "* const ls_tile = (" << T << "*)ls_tsm;\n";
    o << "  __shared__ int s_lo[3], s_hi[3];\n";
    if (fixed) o << "  const float isc = __ldg(a.iscale);\n";
    o << "  const int E0 = a.e0, E1 = a.e1, E2 = a.e2, CS = a.cstride, CU = a.cunit;"
         " (void)E1; (void)E2; (void)CS; (void)CU;\n";
    o << "#define LS_OUT_OF_RANGE(V) { }\n";
    o << "  const long long B = blockDim.x;\n";
    o << "  for (long long t0 = (long long)blockIdx.x * B; t0 < a.n; t0 += (long long)gridDim.x * B) {\n";
    o << "    if (threadIdx.x < 3) { s_lo[threadIdx.x] = 0x7fffffff; s_hi[threadIdx.x] = -0x7fffffff; }\n";
    o << "    __syncthreads();\n";
    o << "    const long long i = t0 + threadIdx.x;\n";
    o << "    float x0 = 0.0f, x1 = 0.0f, x2 = 0.0f, gp = 0.0f;\n    (void)x2;\n";
    o << "    bool good = false;\n";
    o << "    int kk[3] = {0, 0, 0};\n";
    o << "    if (i < a.n) {\n";
    for (int q = 0; q < D; ++q) o << "      x" << q << " = ls_ld_pt(a.pts + (size_t)i * " << D << " + " << q << ");\n";
    o << "      gp = __ldg(a.gout + i);\n";
    o << "      good = gp != 0.0f";
    for (int q = 0; q < D; ++q) o << " && fabsf(x" << q << ") < 4194304.0f";
    o << ";\n    }\n";
    o << "    if (good) {\n" << roe_only(t);
    for (int q = 0; q < D; ++q) o << "      kk[" << q << "] = k" << q << ";\n";
    o << "    }\n";
    for (int q = 0; q < D; ++q) {
        o << "    {\n      int lo = good ? kk[" << q << "] : 0x7fffffff, hi = good ? kk[" << q << "] : -0x7fffffff;\n";
        o << "      lo = __reduce_min_sync(0xffffffffu, lo); hi = __reduce_max_sync(0xffffffffu, hi);\n";
        o << "      if ((threadIdx.x & 31) == 0) { atomicMin(&s_lo[" << q << "], lo); atomicMax(&s_hi[" << q
          << "], hi); }\n    }\n";
    }
    o << "    __syncthreads();\n";
    o << "    int qlo[3] = {0, 0, 0};\n";
    o << "    bool fits = s_lo[0] <= s_hi[0];\n";
    for (int q = 0; q < D; ++q) {
        if (sc == 2) {
            o << "    qlo[" << q << "] = (s_lo[" << q << "] - " << reach << ") >> 1;\n";
            o << "    fits = fits && ((s_hi[" << q << "] + " << reach << ") >> 1) - qlo[" << q << "] < " << TE << ";\n";
        } else {
            o << "    qlo[" << q << "] = s_lo[" << q << "] - " << reach << ";\n";
            o << "    fits = fits && (s_hi[" << q << "] + " << reach << ") - qlo[" << q << "] < " << TE << ";\n";
        }
    }
    o << "    if (fits) {\n";
    o << "      for (int q = threadIdx.x; q < " << TN << "; q += blockDim.x) ls_tile[q] = 0;\n";
    o << "      __syncthreads();\n";
    o << "      if (good) {\n";
    // the tile as an interleaved volume of TE^D grid indices, sites relative to sc * qlo
    o << "      const int ksh0 = " << sc << " * qlo[0], ksh1 = " << sc << " * qlo[1], ksh2 = " << sc
      << " * qlo[2]; (void)ksh1; (void)ksh2;\n";
    o << "      const int E0 = " << TE << ", E1 = " << TE << ", E2 = " << TE << ", CS = 1, CU = " << C
      << "; (void)E1; (void)E2; (void)CS; (void)CU;\n";
    emit_adjoint_body(e, t, st, reach, tadd, "ksh");
    o << "      }\n";
    o << "      __syncthreads();\n";
    // one global add per nonzero tile element inside the arrays
    o << "      for (int q = threadIdx.x; q < " << TN << "; q += blockDim.x) {\n";
    o << "        const " << T << " v = ls_tile[q];\n";
    o << "        if (v == 0) continue;\n";
    o << "        const int j = q % " << C << ", r = q / " << C << ";\n";
    o << "        const int g0 = qlo[0] + r % " << TE << ";\n";
    if (D >= 2) o << "        const int g1 = qlo[1] + (r / " << TE << ") % " << TE << ";\n";
    if (D == 3) o << "        const int g2 = qlo[2] + r / " << TE * TE << ";\n";
    o << "        if (g0 < 0 || g0 >= E0";
    if (D >= 2) o << " || g1 < 0 || g1 >= E1";
    if (D == 3) o << " || g2 < 0 || g2 >= E2";
    o << ") continue;\n";
    o << "        const int ad = j * CS + CU * (g0";
    if (D >= 2) o << " + E0 * (g1";
    if (D == 3) o << " + E1 * g2";
    if (D >= 2) o << ")";
    o << ");\n";
    if (fixed) o << "        atomicAdd(a.iacc + ad, v);\n";
    else o << "        atomicAdd(a.dcoef + ad, v);\n";
    o << "      }\n";
    o << "      __syncthreads();\n";
    o << "    } else if (good) {\n";
    emit_adjoint_body(e, t, st, reach, gadd);
    o << "    }\n";
    o << "  }\n#undef LS_OUT_OF_RANGE\n}\n\n";
    return TN * (fixed ? 8 : 4);
}

// ---------------------------------------------------------------------------
// deterministic adjoint: binning by region-of-evaluation site + per-coefficient gather
// ---------------------------------------------------------------------------

// Offsets d = n - k between a coefficient site n and the region-of-evaluation
// site k of any point whose stencil contains n: all images T^T s_j of the
// stencil sites under the fold group (Cartesian, deduplicated, sorted).
std::vector<I3> reverse_offsets(const Table &t, const Stencil &st)
{
    std::set<I3> out;
    const int D = t.dim;
    std::vector<I3> sites = st.sites;
    if (!t.sep.empty()) {
        sites.clear();
        const int n1 = D > 1 ? (int)t.sep[1].sites.size() : 1, n2 = D > 2 ? (int)t.sep[2].sites.size() : 1;
        for (int j2 = 0; j2 < n2; ++j2)
            for (int j1 = 0; j1 < n1; ++j1)
                for (int s0 : t.sep[0].sites)
                    sites.push_back({s0, D > 1 ? t.sep[1].sites[j1] : 0, D > 2 ? t.sep[2].sites[j2] : 0});
    }
    std::vector<int> perm(D);
    for (int i = 0; i < D; ++i) perm[i] = i;
    do {
        for (int sg = 0; sg < (1 << D); ++sg) {
            for (const auto &s : sites) {
                I3 m{0, 0, 0};
                // m[p_r] = sign * s_r
                for (int r = 0; r < D; ++r) m[perm[r]] = ((sg >> perm[r]) & 1) ? -s[r] : s[r];
                out.insert(m);
            }
            if (t.fold == LS_FOLD_NONE) break;
        }
        if (t.fold == LS_FOLD_NONE) break;
    } while (std::next_permutation(perm.begin(), perm.end()));
    return std::vector<I3>(out.begin(), out.end());
}

int bin_halo(const Table &t, int reach) { return (reach + t.scale - 1) / t.scale + 1; }

void emit_adjoint_bin(Emitter &e, const Table &t, const ls_variant &var)
{
    auto &o = e.o;
    const int D = t.dim;
    o << "extern \"C\" __global__ void __launch_bounds__(" << var.block << ") " << kname(t, "adjoint_bin")
      << "(const LsBinArgs a)\n{\n";
    o << "  const long long stride = (long long)gridDim.x * blockDim.x;\n";
    o << "  const int H = a.halo;\n";
    o << "  const int eb0 = a.e0 + 2 * H, eb1 = a.e1 + 2 * H, eb2 = a.e2 + 2 * H; (void)eb1; (void)eb2;\n";
    o << "#define LS_OUT_OF_RANGE(V) { a.key[i] = a.nbins; a.idx[i] = (int)i; a.rec[i] = make_float4(0.f, 0.f, 0.f, 0.f); }\n";
    o << "  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {\n";
    emit_point_load(e, t);
    o << "    const float gp = __ldg(a.gout + i);\n";
    emit_classify(e, t);
    // bin of k in the haloed grid
    const unsigned long long lut = coset_lut(t);
    if (t.scale == 2) {
        o << "    const int par = (k0 & 1)";
        for (int i = 1; i < D; ++i) o << " | ((k" << i << " & 1) << " << i << ")";
        o << ";\n    const int cid = (int)((" << lut << "ull >> (4 * par)) & 15ull);\n";
        for (int i = 0; i < D; ++i) o << "    const int bi" << i << " = (k" << i << " >> 1) + H;\n";
    } else {
        o << "    const int cid = 0;\n";
        for (int i = 0; i < D; ++i) o << "    const int bi" << i << " = k" << i << " + H;\n";
    }
    o << "    const bool inb = (gp != 0.0f)";
    for (int i = 0; i < D; ++i) o << " && (unsigned)bi" << i << " < (unsigned)eb" << i;
    o << ";\n";
    o << "    const unsigned cs = (unsigned)eb0" << (D > 1 ? " * (unsigned)eb1" : "") << (D > 2 ? " * (unsigned)eb2" : "")
      << ";\n";
    o << "    const unsigned b = (unsigned)cid * cs + (unsigned)bi0";
    if (D > 1) o << " + (unsigned)eb0 * ((unsigned)bi1";
    if (D > 2) o << " + (unsigned)eb1 * (unsigned)bi2";
    if (D > 1) o << ")";
    o << ";\n";
    o << "    a.key[i] = inb ? b : a.nbins;\n    a.idx[i] = (int)i;\n";
    o << "    a.rec[i] = make_float4(y0, " << (D > 1 ? "y1" : "0.f") << ", " << (D > 2 ? "y2" : "0.f") << ", gp);\n";
    o << "  }\n#undef LS_OUT_OF_RANGE\n}\n\n";
}

// Horner of w_j(u) with the site index j known only at run time: coefficients
// read from a shared-memory table laid out monomial-major (cw[off + a*NS + j]).
std::string emit_runtime_horner(Emitter &e, const RefRegion &r, int D, const std::string *uv, int off,
                                const char *jvar)
{
    const int NS = (int)r.sites.size();
    std::map<I3, int> mindex;
    for (size_t a = 0; a < r.mono.size(); ++a) mindex[r.mono[a]] = (int)a;
    std::set<I3> sup(r.mono.begin(), r.mono.end());
    PolyEmit pe{e, D, "", {uv[0], uv[1], D > 2 ? uv[2] : std::string()}, {}, {}};
    auto coef = [&](const I3 &m) -> std::string {
        auto it = mindex.find(m);
        if (it == mindex.end()) return std::string();
        return "cw[" + std::to_string(off + it->second * NS) + " + " + jvar + "]";
    };
    return pe.horner(0, I3{0, 0, 0}, coef, sup);
}

void emit_adjoint_gather(Emitter &e, const Table &t, const ls_variant &var, const Stencil & /*st*/, int reach,
                         const std::vector<I3> &doffs)
{
    auto &o = e.o;
    const int D = t.dim;
    const bool sep = !t.sep.empty();
    const int R = reach, W = 2 * reach + 1;
    int lut_size = 1;
    for (int i = 0; i < D; ++i) lut_size *= W;
    int cw_total = 0;
    std::vector<int> cw_off;
    if (!sep) {
        // LUT: (psi, s) -> j within region psi, or -1
        o << "__constant__ signed char ls_jlut[" << t.ref.size() * lut_size << "] = {";
        for (size_t k = 0; k < t.ref.size(); ++k) {
            std::vector<int> lut(lut_size, -1);
            for (size_t j = 0; j < t.ref[k].sites.size(); ++j) {
                const I3 &s = t.ref[k].sites[j];
                int idx = 0;
                for (int i = 0; i < D; ++i) idx = idx * W + (s[i] + R);
                lut[idx] = (int)j;
            }
            for (int v : lut) o << v << ",";
        }
        o << "};\n";
        for (const auto &r : t.ref) {
            cw_off.push_back(cw_total);
            cw_total += (int)(r.mono.size() * r.sites.size());
        }
        o << "__constant__ int ls_doff[" << 3 * doffs.size() << "] = {";
        for (const auto &d : doffs) o << d[0] << "," << d[1] << "," << d[2] << ",";
        o << "};\n";
        o << "__constant__ float ls_cw[" << cw_total << "] = {";
        for (const auto &r : t.ref) {
            const size_t NS = r.sites.size(), NM = r.mono.size();
            for (size_t a = 0; a < NM; ++a)
                for (size_t j = 0; j < NS; ++j) o << flit(r.coef[j * NM + a]) << ",";
        }
        o << "};\n";
    }
    o << "extern \"C\" __global__ void __launch_bounds__(" << var.block << ") " << kname(t, "adjoint_gather")
      << "(const LsGatherArgs a)\n{\n";
    if (!sep) {
        o << "  __shared__ float cw[" << cw_total << "];\n";
        o << "  __shared__ signed char jlut[" << t.ref.size() * lut_size << "];\n";
        o << "  for (int q = threadIdx.x; q < " << cw_total << "; q += blockDim.x) cw[q] = ls_cw[q];\n";
        o << "  for (int q = threadIdx.x; q < " << t.ref.size() * lut_size << "; q += blockDim.x) jlut[q] = ls_jlut[q];\n";
        o << "  __syncthreads();\n";
    }
    o << "  const int H = a.halo;\n";
    o << "  const int eb0 = a.e0 + 2 * H, eb1 = a.e1 + 2 * H, eb2 = a.e2 + 2 * H; (void)eb1; (void)eb2;\n";
    o << "  const unsigned csb = (unsigned)eb0" << (D > 1 ? " * (unsigned)eb1" : "") << (D > 2 ? " * (unsigned)eb2" : "")
      << ";\n";
    // site = cj * cstride + q * cunit in either layout
    o << "  const long long P = (long long)a.e0 * a.e1 * a.e2;\n";
    o << "  const long long total = P * " << t.cosets.size() << ";\n";
    o << "  for (long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x; site < total;"
         " site += (long long)gridDim.x * blockDim.x) {\n";
    if (e.brick) {
        // bricked: site = C * (brick * BV + within) + cj, within = (i2&1) 4 + (i1&1) 2 + (i0&1)
        const int bv = D == 3 ? 8 : 4;
        o << "    const int cj = (int)(site % " << t.cosets.size() << ");\n";
        o << "    const int w = (int)(site / " << t.cosets.size() << ");\n";
        o << "    const int wi = w & " << bv - 1 << ";\n";
        o << "    int bk = w >> " << (D == 3 ? 3 : 2) << ";\n";
        o << "    const int i0 = (bk % (a.e0 >> 1)) * 2 + (wi & 1); bk /= (a.e0 >> 1);\n";
        if (D > 1) o << "    const int i1 = (bk % (a.e1 >> 1)) * 2 + ((wi >> 1) & 1); bk /= (a.e1 >> 1);\n";
        if (D > 2) o << "    const int i2 = bk * 2 + (wi >> 2);\n";
    } else {
        o << "    const int cj = (int)((site / a.cstride) % " << t.cosets.size() << ");\n";
        o << "    int rem = (int)((site / a.cunit) % P);\n";
        o << "    const int i0 = rem % a.e0; rem /= a.e0;\n";
        if (D > 1) o << "    const int i1 = rem % a.e1; rem /= a.e1;\n";
        if (D > 2) o << "    const int i2 = rem;\n";
    }
    // Cartesian site n
    for (int i = 0; i < D; ++i) {
        o << "    int l" << i << " = 0;\n";
        for (size_t j = 0; j < t.cosets.size(); ++j)
            if (t.cosets[j][i]) o << "    if (cj == " << j << ") l" << i << " = " << t.cosets[j][i] << ";\n";
        o << "    const int nn" << i << " = " << t.scale << " * i" << i << " + l" << i << ";\n";
    }
    o << "    float acc = 0.0f;\n";
    const unsigned long long lut = coset_lut(t);
    // bin of k = n - d and the loop over its points; dexpr[i] is the offset
    // component (an immediate, or a variable read from the offset table)
    auto open_bin_loop = [&](const std::string *dexpr) {
        for (int i = 0; i < D; ++i) o << "      const int kk" << i << " = nn" << i << " - (" << dexpr[i] << ");\n";
        if (t.scale == 2) {
            o << "      const int par = (kk0 & 1)";
            for (int i = 1; i < D; ++i) o << " | ((kk" << i << " & 1) << " << i << ")";
            o << ";\n      const unsigned kc = (unsigned)((" << lut << "ull >> (4 * par)) & 15ull);\n";
            for (int i = 0; i < D; ++i) o << "      const int bi" << i << " = (kk" << i << " >> 1) + H;\n";
        } else {
            o << "      const unsigned kc = 0u;\n";
            for (int i = 0; i < D; ++i) o << "      const int bi" << i << " = kk" << i << " + H;\n";
        }
        o << "      const unsigned b = kc * csb + (unsigned)bi0";
        if (D > 1) o << " + (unsigned)eb0 * ((unsigned)bi1";
        if (D > 2) o << " + (unsigned)eb1 * (unsigned)bi2";
        if (D > 1) o << ")";
        o << ";\n";
        o << "      const unsigned pend = __ldg(a.start + b + 1);\n";
        o << "      for (unsigned pos = __ldg(a.start + b); pos < pend; ++pos) {\n";
        o << "        const float4 r = __ldg(a.srec + pos);\n";
        o << "        const float y0 = r.x" << (D > 1 ? ", y1 = r.y" : "") << (D > 2 ? ", y2 = r.z" : "")
          << ", gp = r.w;\n";
    };
    if (sep) {
        // tensor product: unrolled over the offsets; the weight of offset d is a
        // product of 1D Horner forms with immediate coefficients
        for (const auto &d : doffs) {
            o << "    {\n";
            std::string de[3] = {std::to_string(d[0]), std::to_string(d[1]), std::to_string(d[2])};
            open_bin_loop(de);
            o << "        float w = gp;\n";
            for (int i = 0; i < D; ++i) {
                const Axis &ax = t.sep[i];
                int jj = -1;
                for (size_t q = 0; q < ax.sites.size(); ++q)
                    if (ax.sites[q] == d[i]) jj = (int)q;
                const int nc = ax.degree + 1;
                std::string acc = flit(ax.coef[jj * nc + ax.degree]);
                for (int dd = ax.degree - 1; dd >= 0; --dd)
                    acc = "fmaf(" + acc + ", y" + std::to_string(i) + " - " + flit(ax.center) + ", " +
                          flit(ax.coef[jj * nc + dd]) + ")";
                o << "        w *= " << acc << ";\n";
            }
            o << "        acc += w;\n";
            o << "      }\n    }\n";
        }
    } else {
        // one copy of the body: the offsets come from a table that all threads of
        // a warp read at the same index
        o << "    for (int qd = 0; qd < " << doffs.size() << "; ++qd) {\n";
        for (int i = 0; i < D; ++i) o << "      const int dv" << i << " = ls_doff[3 * qd + " << i << "];\n";
        std::string de[3] = {"dv0", "dv1", "dv2"};
        open_bin_loop(de);
        // fold the point, then s = T d (reference offset of this coefficient)
        o << "        const unsigned ng0 = y0 < 0.0f" << (D > 1 ? ", ng1 = y1 < 0.0f" : "")
          << (D > 2 ? ", ng2 = y2 < 0.0f" : "") << ";\n";
        if (t.fold == LS_FOLD_SIGNED_PERM) {
            for (int i = 0; i < D; ++i)
                o << "        float a" << i << " = fabsf(y" << i << "); int p" << i << " = " << i << "; unsigned g" << i
                  << " = ng" << i << ";\n";
            if (D == 3)
                o << "        LS_CSWAP(a0, a1, p0, p1, g0, g1); LS_CSWAP(a1, a2, p1, p2, g1, g2);"
                     " LS_CSWAP(a0, a1, p0, p1, g0, g1);\n";
            else
                o << "        LS_CSWAP(a0, a1, p0, p1, g0, g1);\n";
            for (int r = 0; r < D; ++r) {
                o << "        const int dr" << r << " = ";
                for (int i = 0; i < D - 1; ++i) o << "(p" << r << " == " << i << ") ? dv" << i << " : ";
                o << "dv" << (D - 1) << ";\n";
                o << "        const int s" << r << " = g" << r << " ? -dr" << r << " : dr" << r << ";\n";
            }
        } else {
            for (int i = 0; i < D; ++i) o << "        const float a" << i << " = y" << i << ";\n";
            for (int r = 0; r < D; ++r) o << "        const int s" << r << " = dv" << r << ";\n";
        }
        if (t.ref.size() > 1) {
            o << "        unsigned q = 0u;\n";
            for (size_t pi = 0; pi < t.planes.size(); ++pi) {
                o << "        q |= (";
                for (int i = 0; i < D; ++i) o << (i ? " + " : "") << flit(t.planes[pi][i]) << " * a" << i;
                o << " - " << flit(t.planes[pi][3]) << " >= 0.0f) ? " << (1u << pi) << "u : 0u;\n";
            }
            unsigned long long packed = 0;
            for (int qq = 0; qq < t.bsp_mod; ++qq) {
                unsigned v = t.sigma[qq] < 0 ? 0u : (unsigned)t.sigma[qq];
                packed |= (unsigned long long)(v & 0xF) << (4 * qq);
            }
            o << "        const int psi = (int)((" << packed << "ull >> (4u * (q % " << t.bsp_mod << "u))) & 15ull);\n";
        } else {
            o << "        const int psi = 0;\n";
        }
        o << "        bool inr = true;\n";
        for (int r = 0; r < D; ++r) o << "        inr = inr && (s" << r << " >= " << -R << ") && (s" << r << " <= " << R << ");\n";
        o << "        if (!inr) continue;\n";
        {
            std::string li = "(s0 + " + std::to_string(R) + ")";
            for (int r = 1; r < D; ++r)
                li = "(" + li + " * " + std::to_string(W) + " + (s" + std::to_string(r) + " + " + std::to_string(R) + "))";
            o << "        const int li = " << li << ";\n";
        }
        o << "        const int jj = jlut[psi * " << lut_size << " + li];\n";
        o << "        if (jj < 0) continue;\n";
        for (size_t k = 0; k < t.ref.size(); ++k) {
            o << "        " << (k ? "else " : "") << "if (psi == " << k << ") {\n";
            std::string uv[3];
            for (int i = 0; i < D; ++i) {
                uv[i] = "v" + std::to_string(k) + "_" + std::to_string(i);
                o << "        const float " << uv[i] << " = a" << i << " - " << flit(t.ref[k].center[i]) << ";\n";
            }
            std::string w = emit_runtime_horner(e, t.ref[k], D, uv, cw_off[k], "jj");
            o << "        acc = fmaf(gp, " << (w.empty() ? "0.0f" : w) << ", acc);\n";
            o << "        }\n";
        }
        o << "      }\n    }\n";
    }
    o << "    a.dcoef[site] += acc;\n";
    o << "  }\n}\n\n";
}

// A bound on |w_j(u)| over the region of evaluation, for the fixed-point adjoint's
// scale: sum_a |M[j][a]| prod_i R_i^{a_i} with R_i = |center_i| + the radius of
// the region (1 for the parallelepiped [0,1)^s; half the sum of the generator's
// column lengths for the Voronoi cell, which holds every point within that
// distance of the site found by rounding in the lattice basis).
double weight_bound(const Table &t)
{
    const int D = t.dim;
    double rad = 1.0;
    if (t.roe == LS_ROE_VORONOI) {
        rad = 0.0;
        for (int j = 0; j < D; ++j) {
            double n2 = 0.0;
            for (int i = 0; i < D; ++i) n2 += t.L[3 * j + i] * t.L[3 * j + i];
            rad += 0.5 * std::sqrt(n2);
        }
        rad = std::max(rad, 1.0);
    }
    double wmax = 0.0;
    if (!t.sep.empty()) {
        wmax = 1.0;
        for (const auto &ax : t.sep) {
            const double R = rad + std::fabs(ax.center);
            double m = 0.0;
            for (size_t j = 0; j < ax.sites.size(); ++j) {
                double b = 0.0, p = 1.0;
                for (int d = 0; d <= ax.degree; ++d, p *= R) b += std::fabs(ax.coef[j * (ax.degree + 1) + d]) * p;
                m = std::max(m, b);
            }
            wmax *= m;
        }
        return wmax;
    }
    for (const auto &r : t.ref) {
        const size_t nm = r.mono.size();
        for (size_t j = 0; j < r.sites.size(); ++j) {
            double b = 0.0;
            for (size_t a = 0; a < nm; ++a) {
                double p = std::fabs(r.coef[j * nm + a]);
                for (int i = 0; i < D; ++i) p *= std::pow(rad + std::fabs(r.center[i]), r.mono[a][i]);
                b += p;
            }
            wmax = std::max(wmax, b);
        }
    }
    return wmax;
}

}  // namespace

Generated generate(const Table &t, ls_dtype dt, const ls_variant &var)
{
    Generated g;
    Emitter e;
    e.ld = loader_name(dt);
    e.brick = var.brick != 0;
    setup_brick_shift(e, t, var.brick, dt);
    e.sym = !var.plain_transform;
    if (var.wait_limit > 0) e.wait_rounds = var.wait_limit;
    e.no_signal = var.wait_probe == 1;
    e.l2_keep = var.l2_keep == 1;
    e.fma2 = var.fma2 == 1;
    emit_prologue(e);
    const size_t tab_at = e.o.str().size();    // the paired transform's constant tables go here
    Stencil st = union_stencil(t);
    int reach = 0;
    if (t.sep.empty()) {
        for (auto &s : st.sites)
            for (int i = 0; i < t.dim; ++i) reach = std::max(reach, std::abs(s[i]));
        g.info.n_sites = (int)st.sites.size();
    } else {
        int n = 1;
        for (auto &ax : t.sep) {
            n *= (int)ax.sites.size();
            for (int s : ax.sites) reach = std::max(reach, std::abs(s));
        }
        g.info.n_sites = n;
    }
    g.info.reach = reach;
    if (var.tensor && t.sep.empty()) {
        emit_eval_point(e, t, var, st, reach, false, kname(t, "eval_pt"));
        emit_eval_kernel_tensor(e, t, var, st, reach, g.info);
    } else if (var.stage && t.dim == 3) {
        g.info.eval_smem = emit_eval_kernel_staged(e, t, var, st, reach, g.info);
    } else if (var.producers > 0 && t.sep.empty()) {
        emit_eval_point(e, t, var, st, reach, false, kname(t, "eval_pt"));
        g.info.eval_smem = emit_eval_kernel_ws(e, t, var, st, reach, g.info);
    } else if (var.pipeline && t.sep.empty()) {
        // the point function still serves batched kernels
        emit_eval_point(e, t, var, st, reach, false, kname(t, "eval_pt"));
        emit_eval_kernel_pipelined(e, t, var, st, reach, g.info);
    } else if (var.pts_per_thread > 1 && t.sep.empty()) {
        // the point function is still emitted (batched kernels, gradient) but the
        // value kernel walks runs of consecutive points
        GenInfo tmp;
        emit_eval_point(e, t, var, st, reach, false, kname(t, "eval_pt"));
        emit_eval_kernel_reuse(e, t, var, st, reach, var.pts_per_thread, g.info);
        (void)tmp;
    } else {
        emit_eval_kernel(e, t, var, st, reach, false, g.info);
    }
    if (var.tensor && t.sep.empty()) emit_eval_kernel_tensor(e, t, var, st, reach, g.info, true);
    else emit_eval_kernel(e, t, var, st, reach, true, g.info);
    {
        const int fma0 = e.fma;
        const std::string pf = kname(t, "eval_hess_pt");
        emit_eval_point_hess(e, t, var, st, reach, pf);
        e.o << "extern \"C\" __global__ void __launch_bounds__(" << var.block << ") " << kname(t, "eval_hess")
            << "(const LsEvalArgs a)\n{\n";
        e.o << "  const long long stride = (long long)gridDim.x * blockDim.x;\n";
        e.o << "  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) " << pf
            << "(a, i);\n}\n\n";
        g.info.fma_hess = e.fma - fma0;
    }
    emit_adjoint_atomic(e, t, var, st, reach, ADJ_ATOMIC);
    emit_adjoint_atomic(e, t, var, st, reach, ADJ_WARPAGG);
    emit_adjoint_atomic(e, t, var, st, reach, ADJ_FIXED);
    g.info.adj_tile_smem = emit_adjoint_tiled(e, t, var, st, reach, false);
    g.info.adj_tile_fixed_smem = emit_adjoint_tiled(e, t, var, st, reach, true);
    g.info.wmax = weight_bound(t);
    emit_adjoint_bin(e, t, var);
    std::vector<I3> doffs = reverse_offsets(t, st);
    emit_adjoint_gather(e, t, var, st, reach, doffs);
    g.info.n_reverse = (int)doffs.size();
    g.info.halo = bin_halo(t, reach);
    g.source = e.o.str();
    g.source.insert(tab_at, e.ktabs);
    return g;
}

Generated generate_batch(const std::vector<const Table *> &tables, const std::vector<ls_dtype> &dts,
                         const std::vector<int> &bricks, const ls_variant &var)
{
    Generated g;
    Emitter e;
    e.fma2 = var.fma2 == 1;
    emit_prologue(e);
    const size_t tab_at = e.o.str().size();
    for (size_t k = 0; k < tables.size(); ++k) {
        const Table &t = *tables[k];
        e.ld = loader_name(dts[k]);
        e.brick = bricks[k] != 0;
        setup_brick_shift(e, t, bricks[k], dts[k]);
        Stencil st = union_stencil(t);
        int reach = 0;
        if (t.sep.empty()) {
            for (auto &sv : st.sites)
                for (int i = 0; i < t.dim; ++i) reach = std::max(reach, std::abs(sv[i]));
        } else {
            for (auto &ax : t.sep)
                for (int sv : ax.sites) reach = std::max(reach, std::abs(sv));
        }
        emit_eval_point(e, t, var, st, reach, false, "ls_bpt_" + std::to_string(k));
    }
    auto &o = e.o;
    o << "struct LsBatchVol { const float* pts; float* out; const void* coef; long long n;"
         " int e0, e1, e2, cstride, kind, cunit; };\n";
    o << "struct LsBatchItem { int vol; int pad; long long p0, p1; };\n";
    o << "struct LsBatchArgs { const LsBatchVol* vols; const LsBatchItem* items; int nitems; int pad;"
         " unsigned* counter; unsigned* status; };\n";
    o << "// Persistent launch: every block takes (volume, tile) items from the list by an\n"
         "// atomic ticket until the list is exhausted; nothing waits on anything.\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << var.block << ") ls_batch_eval(const LsBatchArgs b)\n{\n";
    o << "  __shared__ int s_item;\n";
    o << "  for (;;) {\n";
    o << "    if (threadIdx.x == 0) s_item = (int)atomicAdd(b.counter, 1u);\n";
    o << "    __syncthreads();\n";
    o << "    const int it = s_item;\n";
    o << "    __syncthreads();\n";
    o << "    if (it >= b.nitems) {\n";
    o << "      // exit ticket: the last block out resets both counters for the next launch\n";
    o << "      if (threadIdx.x == 0) {\n";
    o << "        __threadfence();\n";
    o << "        const unsigned d = atomicAdd(b.counter + 1, 1u);\n";
    o << "        if (d == gridDim.x - 1) { atomicExch(b.counter, 0u); atomicExch(b.counter + 1, 0u); }\n";
    o << "      }\n";
    o << "      return;\n";
    o << "    }\n";
    o << "    const LsBatchItem w = b.items[it];\n";
    o << "    const LsBatchVol v = b.vols[w.vol];\n";
    o << "    LsEvalArgs a;\n";
    o << "    a.pts = v.pts; a.out = v.out; a.grad = 0; a.coef = v.coef; a.n = v.n;\n";
    o << "    a.e0 = v.e0; a.e1 = v.e1; a.e2 = v.e2; a.cstride = v.cstride; a.cunit = v.cunit; a.status = b.status;"
         " a.hess = 0; a.tmap = 0;\n";
    o << "    switch (v.kind) {\n";
    for (size_t k = 0; k < tables.size(); ++k)
        o << "    case " << k << ": for (long long i = w.p0 + threadIdx.x; i < w.p1; i += blockDim.x) ls_bpt_" << k
          << "(a, i); break;\n";
    o << "    default: if (threadIdx.x == 0) atomicOr(b.status, 1u); break;\n";
    o << "    }\n  }\n}\n";
    g.source = e.o.str();
    g.source.insert(tab_at, e.ktabs);
    return g;
}

}  // namespace ls
