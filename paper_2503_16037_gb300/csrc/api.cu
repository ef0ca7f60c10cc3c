// C ABI of libtursca_gb (declared in include/tursca.h): scene lifecycle,
// uploads, stage orchestration and the solver control loop.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <functional>
#include <vector>

#include "graph.h"
#include "first_order.h"
#include "kern.h"
#include "batch.h"
#include "select.h"
#include "aniso.h"
#include "tursca.h"

namespace {
thread_local std::string g_last_error;
}

// device allocations owned by a scene, with their total size
struct AllocList {
    std::vector<void *> ptrs;
    size_t bytes = 0;
};

// a device buffer reused across calls, grown only when a call needs more
// (a geometry change then costs no device-wide synchronisation of cudaFree)
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

// GMRES is right-preconditioned with the Neumann polynomial
// M^-1 = I + K + ... + K^(kGmresPoly - 1) (1: no preconditioning; the
// truncated series of Eq. fs_sum).  Measured on GB300: degree 2 (I + K) takes
// the broken cloud from 46.2 to 37.5 ms and the FP64 plume from 6.45 to
// 5.40 ms; degrees 3 and 4 spend more in products than they save in steps.
#ifndef TK_GMRES_POLY
#define TK_GMRES_POLY 2
#endif
constexpr int kGmresPoly = TK_GMRES_POLY;
// restart length of GMRES on FP32 scenes (FP64 scenes: 40); measured on the
// broken cloud: 20 / 30 / 40 gave 39.4 / 37.4 / 38.1 ms
#ifndef TK_GMRES_M32
#define TK_GMRES_M32 30
#endif

// one geometry-dependent device buffer per slot
enum VSlot {
    VB_SUN_TAPS, VB_SUN_LF, VB_SUN_LD, VB_SUN_OFF, VB_SUN_N, VB_SUN_RT,
    VB_LOS_TAPS, VB_LOS_LF, VB_LOS_LD, VB_LOS_OFF, VB_LOS_N,
    VB_PIX_CX, VB_PIX_CY, VB_PIX_CLS, VB_RAD, VB_REFL, VB_COUNT
};

struct tursca_scene {
    tursca_grid_desc d{};
    cudaStream_t st = nullptr;
    std::string err;
    long long launches = 0;
    size_t es = 4;  // element size of the compute type

    tg::Graph G;
    bool built = false;
    tg::ViewTables VT;
    bool view_ok = false;
    tursca_geometry geom{};
    bool medium = false, assembled = false, solved = false, rendered = false;
    // adjoint state (allocated on the first tursca_adjoint)
    bool adj_ready = false;
    int *tstartT = nullptr, *flatT = nullptr, *hgdirT = nullptr;
    long long *voffT = nullptr;
    int4 *infoT = nullptr;
    void *valT = nullptr, *Lbar = nullptr;
    double *lam64 = nullptr;
    void *adj[10] = {nullptr};  // Ebar, Ebar_h, e1bar, e1bar_h, xbar, mubar, mubar_h, tsegbar, tinfbar, tinfgbar
    size_t adj_bytes[10] = {0};
    double g[tk::MAX_SPECIES] = {0, 0, 0, 0};
    double albedo = 0.0;

    AllocList allocs;       // graph-lifetime allocations
    DevBuf vbuf[VB_COUNT];  // geometry-dependent buffers (sun and line-of-sight taps, pixels, images)

    // graph
    int *tstart = nullptr;
    int4 *tmpl = nullptr;
    long long *voff = nullptr;
    tk::DClass *cls = nullptr;
    tk::DTap *taps = nullptr;
    float *tlf = nullptr;
    double *tld = nullptr;
    int4 *dirs = nullptr, *gmem1 = nullptr;
    double *dir_len = nullptr, *q_iso = nullptr, *q_lamb = nullptr, *gdist1 = nullptr;
    float *dir_len_f = nullptr, *q_iso_f = nullptr, *q_lamb_f = nullptr, *gdist1_f = nullptr;
    int *up_dirs = nullptr, *top_off = nullptr, *top_n = nullptr, *lat_off = nullptr, *lat_n = nullptr,
        *gtop_off = nullptr, *gtop_n = nullptr;
    double *lattice = nullptr, *dirhat = nullptr;
    int *cell_start = nullptr;
    int *canon_dirs = nullptr, *up_canon = nullptr;
    int4 *cseg = nullptr;   // per canonical direction: (first tap in ctap, tap count, u_z, 0)
    int *ctap = nullptr;    // graph tap index of each tap of the canonical segments
    int nctap = 0;
    tk::SegTab<float> segtab_f;   // the canonical segments as kernel parameters (n = 0: not used)
    tk::SegTab<double> segtab_d;
    void *srec = nullptr;   // source records of the edge kernel (haloed, srec_stride(S) per node)
    int *tflat = nullptr;  // template offsets in the haloed layout
    tk::RTap *rtaps = nullptr, *sun_rt = nullptr;  // taps of long rays, pre-wrapped (graph, sun)
    int *ttile = nullptr, *tlay = nullptr;  // gather-tile offsets and layers of the row-group passes
    int tile_tl = 0;                        // floats per tile layer (0: no tiles)
    int *ttileT = nullptr, *tlayT = nullptr;  // the same for the K^T passes of the adjoint
    int tile_tlT = 0;
    tk::ASlot *aslot = nullptr;  // edge-kernel descriptors of the template entries
    int *tap_h = nullptr, *dir_h = nullptr;  // haloed offsets of the taps and the directions
    void *rt_h = nullptr, *wsp_h = nullptr, *mu_e_h = nullptr, *e1_h = nullptr;  // haloed copies
    void *mu_x = nullptr;  // extinction repeated 2 x 2 horizontally (long rays)
    int *run_g[2] = {nullptr, nullptr};  // runs of the persistent streamed passes
    long long *run_v[2] = {nullptr, nullptr};
    int run_n[2] = {0, 0};
    // view
    tk::DTap *sun_taps = nullptr, *los_taps = nullptr;
    float *sun_lf = nullptr, *los_lf = nullptr;
    double *sun_ld = nullptr, *los_ld = nullptr;
    int *sun_off = nullptr, *sun_n = nullptr, *los_off = nullptr, *los_n = nullptr, *pix_cx = nullptr,
        *pix_cy = nullptr, *pix_cls = nullptr;
    void *rad = nullptr, *refl = nullptr;
    // fields (compute type)
    void *mu_a = nullptr, *mu_s = nullptr, *mu_e = nullptr, *mu_st = nullptr, *tsun = nullptr, *e1 = nullptr,
         *tinf = nullptr, *tinfg = nullptr, *zc_iso = nullptr, *zc_sun = nullptr, *tseg = nullptr, *rt = nullptr, *wsp = nullptr, *q_sun = nullptr, *hgv = nullptr,
         *hg0v = nullptr, *val = nullptr, *s = nullptr, *gsun = nullptr, *emis = nullptr;
    unsigned long long *musmax = nullptr;
    int *status = nullptr;
    double *cellsum = nullptr;
    bool fields_alloc = false;
    // solver
    double *x64 = nullptr, *r64 = nullptr, *part = nullptr, *dred = nullptr, *hred = nullptr;
    void *b = nullptr, *d0 = nullptr, *d1 = nullptr, *V = nullptr, *w = nullptr;
    float *xh = nullptr, *xl = nullptr;  // double-single split of x
    int gm_m = 0;
    int resid_fp64 = 0;  // 1: evaluate the refinement residual with FP64 arithmetic
    int stage_values = 0;  // 1: FP32 passes stream the values through shared memory (persistent kernels)
    int l2_resident = 0;   // 1: the solves keep the values of K in the persisting part of L2
    int gather_tile = 1;   // 1: FP32 passes gather from a shared-memory tile
    int single = 0;        // 1: the next assembly takes the first scattering order only
    // coupling selection (c_min > 0): lattice rankings, per-scene buffers and
    // the weight planes of every (source, direction)
    double c_min = 0.0;
    // the preselected maximum number of couplings (0: off) and the state of
    // its selection: per-chain keys, the radix histogram, the last threshold,
    // the number of chains with a receiver
    long long max_couplings = 0;
    // the serving loop's batcher of Chebyshev refinements (null: own passes)
    tk::ChebBatcher *batcher = nullptr;
    cudaEvent_t bready = nullptr, bdone = nullptr;
    unsigned long long *topk_keys = nullptr;
    unsigned int *topk_hist = nullptr, *topk_hist_h = nullptr;
    int *topk_band = nullptr, *topk_cnt = nullptr;  // chains in the FP32 band, [2] listed / above
    double c_eff = 0.0;
    long long n_couplings = -1, n_kept = -1;
    bool sel_ready = false, sel_asm = false;
    tk::SelP selp{};
    void *w_iso = nullptr, *w_sun = nullptr;
    // anisotropic multiple scattering (edge unknowns): option, state, buffers
    int aniso = 0;
    bool aniso_asm = false, ani_ready = false;
    void *ani_Q = nullptr, *ani_SQ = nullptr, *ani_CT = nullptr, *ani_on = nullptr, *ani_zf = nullptr,
         *ani_LsT = nullptr, *ani_Wg = nullptr, *ani_Lh = nullptr, *ani_X = nullptr, *ani_Xn = nullptr;
    double *ani_Qraw = nullptr, *ani_acc = nullptr, *ani_part = nullptr;
    int *ani_ctl = nullptr;
    int4 *ani_tslot = nullptr;  // slots of each layer by arrival direction (graph build): {t, src, dir, 0}
    int *ani_tseg = nullptr;    // start of each arrival direction's run
    int ani_max_nt = 0;         // slots of the largest layer template
    float *ani_Bl = nullptr;                          // tensor-core operand (FP32 scenes)
    void *ani_CfH = nullptr, *ani_Pc = nullptr, *ani_b = nullptr;  // the series' folded form
    void *ani_xtg = nullptr, *ani_xtb = nullptr;                   // ground nodes' sums of X and of b
    void *ani_Xsol = nullptr;  // the solved X: FP32 pairs (FP32 scenes) or FP64, [nin][ldx]; null before a solve
    bool ani_tables = false;                  // the quadrature tables hold ani_g's asymmetries
    // the node form's quadrature tables (q^sun, HG weights toward the
    // instrument) hold the view and asymmetries in qt_key (sun and view
    // directions, then g per species)
    bool qt_ok = false;
    double qt_key[6 + tk::MAX_SPECIES] = {0.0};
    double ani_g[tk::MAX_SPECIES] = {0.0};
    float2 *ani_X64 = nullptr, *ani_L64 = nullptr;    // FP32 refinement: X and the leaving power in FP32 pairs
    float *ani_r = nullptr, *ani_E = nullptr;         // FP32 refinement: residual, correction
    float2 *ani_Ads = nullptr, *ani_Atop = nullptr;   // FP32 refinement: split operands of the residual
    float *ani_Bds = nullptr;
    bool single_asm = false;  // the current assembly is first-order only (no K, s = 0, x = 0)
    int wq = 8;          // warps per 128-row group of the row-group passes
    bool wq_auto = true;  // wq chosen by the library (else set by the caller)
    // auxiliary streams and events for the concurrent per-scene tables
    cudaStream_t aux[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t fork[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // event timing of the hot kernels
    bool prof = false;
    std::vector<cudaEvent_t> ev;   // pairs
    std::vector<int> ev_cat;
    std::vector<int> ev_n;         // launches covered by each pair
    size_t ev_used = 0;
};

namespace {
const char *const kProfNames[] = {"spmv",   "resid64",    "assemble_rows", "assemble_pre",  "render",
                                  "cheb",   "gmres_orth", "select",        "gmres_prod",    "set_medium",
                                  "solve",  "ani_leave",  "ani_transport", "ani_residual"};
constexpr int kNProf = 14;
// P_GPROD: the passes over K of one Arnoldi step (preconditioner and product
// with I - K), counted as launches; P_MEDIUM: the copies of set_medium;
// P_SOLVE: a whole solve, from its first to its last operation on the stream
// (the other categories of the solve lie inside it); P_ALEAVE, P_AMOVE: the
// edge form's per-term leaving power (contraction and ground) and transport
// (with its stopping test), terms past convergence included; P_ARESID: a
// whole residual evaluation of its refinement
enum {
    P_SPMV = 0, P_RESID = 1, P_ROWS = 2, P_PRE = 3, P_RENDER = 4, P_CHEB = 5, P_ORTH = 6, P_SEL = 7, P_GPROD = 8,
    P_MEDIUM = 9, P_SOLVE = 10, P_ALEAVE = 11, P_AMOVE = 12, P_ARESID = 13
};

// NVTX range around one call of the C ABI (a stage of the path), for
// profilers that filter or group by range; free when no tool is attached
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// returns the index of the pair, or -1 when profiling is off
int prof_begin(tursca_scene *sc, int cat) {
    if (!sc->prof) return -1;
    if (sc->ev_used * 2 + 2 > sc->ev.size()) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            sc->ev.push_back(e);
        }
        sc->ev_cat.resize(sc->ev.size() / 2);
        sc->ev_n.resize(sc->ev.size() / 2);
    }
    size_t i = sc->ev_used++;
    sc->ev_cat[i] = cat;
    sc->ev_n[i] = 1;
    cudaEventRecord(sc->ev[2 * i], sc->st);
    return (int)i;
}
// n: launches of the category between the pair (a run of back-to-back
// launches of one kernel is timed as a whole, so that the events do not
// break the overlap of consecutive launches)
void prof_end(tursca_scene *sc, int i, int n = 1) {
    if (i < 0) return;
    sc->ev_n[i] = n;
    cudaEventRecord(sc->ev[2 * i + 1], sc->st);
}
}  // namespace

namespace {

tursca_status fail(tursca_scene *sc, tursca_status code, const std::string &msg) {
    if (sc) sc->err = msg;
    g_last_error = msg;
    return code;
}

tursca_status cuda_fail(tursca_scene *sc, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(sc, e == cudaErrorMemoryAllocation ? TURSCA_E_NOMEM : TURSCA_E_CUDA, m);
}

#define CK(expr, where)                                   \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) return cuda_fail(sc, _e, where); \
    } while (0)

template <typename P>
cudaError_t dalloc(AllocList &list, P *&p, size_t bytes) {
    void *q = nullptr;
    const size_t b = bytes ? bytes : 16;
    cudaError_t e = cudaMalloc(&q, b);
    if (e != cudaSuccess) return e;
    list.ptrs.push_back(q);
    list.bytes += b;
    p = reinterpret_cast<P *>(q);
    return cudaSuccess;
}

template <typename P>
cudaError_t upload(tursca_scene *sc, AllocList &list, P *&p, const void *src, size_t bytes) {
    cudaError_t e = dalloc(list, p, bytes);
    if (e != cudaSuccess) return e;
    if (bytes) e = cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, sc->st);
    return e;
}

void free_list(AllocList &list) {
    for (void *p : list.ptrs) cudaFree(p);
    list.ptrs.clear();
    list.bytes = 0;
}

// copy bytes from host src into buffer b (grown if needed) on stream st
template <typename P>
cudaError_t put(DevBuf &b, P *&out, const void *src, size_t bytes, cudaStream_t st) {
    const size_t need = bytes ? bytes : 16;
    if (need > b.cap) {
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
        cudaError_t e = cudaMalloc(&b.p, need);
        if (e != cudaSuccess) return e;
        b.cap = need;
    }
    out = reinterpret_cast<P *>(b.p);
    return (bytes && src) ? cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
}

tk::GridC grid_c(const tursca_scene *sc) {
    const tg::Graph &G = sc->G;
    tk::GridC g;
    g.nx = sc->d.nx;
    g.ny = sc->d.ny;
    g.nz = sc->d.nz;
    g.nxy = g.nx * g.ny;
    g.n_atm = g.nxy * g.nz;
    g.n_ground = g.nxy;
    g.n_nodes = g.n_atm + g.n_ground;
    g.S = sc->d.n_species;
    g.nd = (int)G.dirs.size();
    g.ngd = (int)G.gdirs.size();
    g.nup = (int)G.up_dirs.size();
    g.R = sc->d.stencil_radius;
    g.nc = (int)G.canon_dirs.size();
    g.wq = sc->wq;
    g.wq_em = sc->wq_auto ? (sc->stage_values && sc->d.precision != TURSCA_FP64 ? 16 : 6) : sc->wq;
    g.gpl = (g.nxy + tk::kGroup - 1) / tk::kGroup;
    g.ntmax = G.max_row;
    g.H = sc->d.stencil_radius;
    g.nxp = g.nx + 2 * g.H;
    g.nyp = g.ny + 2 * g.H;
    g.lp = g.nxp * g.nyp;
    g.npad = (long long)(g.nz + 1) * g.lp;
    g.stage = (sc->stage_values && sc->d.precision != TURSCA_FP64 && tk::stage_fits(G.max_row)) ? 1 : 0;
    g.tl = sc->gather_tile ? sc->tile_tl : 0;
    g.hx = sc->d.hx;
    g.hy = sc->d.hy;
    g.hz = sc->d.hz;
    return g;
}

tk::GraphP graph_p(const tursca_scene *sc) {
    tk::GraphP p;
    p.tstart = sc->tstart;
    p.tmpl = sc->tmpl;
    p.voff = sc->voff;
    p.cls = sc->cls;
    p.taps = sc->taps;
    p.tap_len_f = sc->tlf;
    p.tap_len_d = sc->tld;
    p.dirs = sc->dirs;
    p.dir_len = sc->dir_len;
    p.q_iso = sc->q_iso;
    p.q_lamb = sc->q_lamb;
    p.q_iso_f = sc->q_iso_f;
    p.q_lamb_f = sc->q_lamb_f;
    p.dir_len_f = sc->dir_len_f;
    p.gdist1_f = sc->gdist1_f;
    p.gmem1 = sc->gmem1;
    p.gdist1 = sc->gdist1;
    p.up_dirs = sc->up_dirs;
    p.top_off = sc->top_off;
    p.top_n = sc->top_n;
    p.lat_off = sc->lat_off;
    p.lat_n = sc->lat_n;
    p.gtop_off = sc->gtop_off;
    p.gtop_n = sc->gtop_n;
    p.rtaps = sc->rtaps;
    p.canon_dirs = sc->canon_dirs;
    p.cseg = sc->cseg;
    p.ctap = sc->ctap;
    p.nctap = sc->nctap;
    p.up_canon = sc->up_canon;
    p.status = sc->status;
    p.tflat = sc->tflat;
    p.ttile = sc->ttile;
    p.tlay = sc->tlay;
    p.aslot = sc->aslot;
    p.tap_h = sc->tap_h;
    p.dir_h = sc->dir_h;
    for (int k = 0; k < 2; ++k) {
        p.run_g[k] = sc->run_g[k];
        p.run_v[k] = sc->run_v[k];
        p.run_n[k] = sc->run_n[k];
    }
    return p;
}

template <typename T>
tk::FieldP<T> field_p(const tursca_scene *sc) {
    tk::FieldP<T> f;
    f.mu_a = (const T *)sc->mu_a;
    f.mu_s = (const T *)sc->mu_s;
    f.mu_e = (T *)sc->mu_e;
    f.mu_st = (T *)sc->mu_st;
    f.tsun = (T *)sc->tsun;
    f.e1 = (T *)sc->e1;
    f.tinf = (T *)sc->tinf;
    f.tinfg = (T *)sc->tinfg;
    f.a_iso = (T *)sc->zc_iso;
    f.a_sun = (T *)sc->zc_sun;
    f.tseg = (T *)sc->tseg;
    f.rt = (T *)sc->rt;
    f.wsp = (T *)sc->wsp;
    f.rt_h = (T *)sc->rt_h;
    f.wsp_h = (T *)sc->wsp_h;
    f.mu_e_h = (T *)sc->mu_e_h;
    f.mu_x = (T *)sc->mu_x;
    f.e1_h = (T *)sc->e1_h;
    f.q_sun = (T *)sc->q_sun;
    f.hgv = (T *)sc->hgv;
    f.hg0v = (T *)sc->hg0v;
    f.val = (T *)sc->val;
    f.s = (T *)sc->s;
    f.gsun = (T *)sc->gsun;
    f.mus_max_bits = sc->musmax;
    f.status = sc->status;
    f.cellsum = sc->cellsum;
    f.srec = (T *)sc->srec;
    return f;
}

tk::ViewC view_c(const tursca_scene *sc) {
    tk::ViewC v;
    for (int a = 0; a < 3; ++a) {
        v.s0[a] = sc->VT.s0[a];
        v.v[a] = sc->VT.v[a];
    }
    v.mu0 = sc->VT.mu0;
    v.f0 = sc->geom.f0;
    v.albedo = sc->albedo;
    for (int s = 0; s < tk::MAX_SPECIES; ++s) v.g[s] = sc->g[s];
    v.coupling = sc->d.coupling_mode;
    return v;
}

tk::ViewP view_p(const tursca_scene *sc) {
    tk::ViewP p;
    p.sun_taps = sc->sun_taps;
    p.sun_rt = sc->sun_rt;
    p.sun_len_f = sc->sun_lf;
    p.sun_len_d = sc->sun_ld;
    p.sun_off = sc->sun_off;
    p.sun_n = sc->sun_n;
    p.los_taps = sc->los_taps;
    p.los_len_f = sc->los_lf;
    p.los_len_d = sc->los_ld;
    p.los_off = sc->los_off;
    p.los_n = sc->los_n;
    p.pix_cx = sc->pix_cx;
    p.pix_cy = sc->pix_cy;
    p.pix_cls = sc->pix_cls;
    p.lattice = sc->lattice;
    p.cell_start = sc->cell_start;
    p.dirhat = sc->dirhat;
    p.npx = sc->geom.npx;
    p.npy = sc->geom.npy;
    return p;
}

void split_taps(const std::vector<tg::Tap> &t, std::vector<tk::DTap> &off, std::vector<float> &lf,
                std::vector<double> &ld) {
    off.resize(t.size());
    lf.resize(t.size());
    ld.resize(t.size());
    for (size_t i = 0; i < t.size(); ++i) {
        off[i] = tk::DTap{(int16_t)t[i].dx, (int16_t)t[i].dy, (int16_t)t[i].dz, 0};
        lf[i] = (float)t[i].len;
        ld[i] = t[i].len;
    }
}

// taps of long rays as RTaps for an nx x ny grid (false: a column offset or
// a layer offset does not fit)
bool ray_taps(const std::vector<tg::Tap> &t, int nx, int ny, std::vector<tk::RTap> &out) {
    if (nx > 0xffff || ny > 0x7fff) return false;
    const long long nxy = (long long)nx * ny;
    out.resize(t.size());
    for (size_t i = 0; i < t.size(); ++i) {
        const int dx = ((t[i].dx % nx) + nx) % nx, dy = ((t[i].dy % ny) + ny) % ny;
        const long long zo = (long long)t[i].dz * nxy;
        if (zo < -(1LL << 31) || zo >= (1LL << 31)) return false;
        out[i] = tk::RTap{dx | (dy << 16), (int)zo};
    }
    return true;
}

std::string check_desc(const tursca_grid_desc *d) {
    if (!d) return "null descriptor";
    if (d->n_species < 1 || d->n_species > tk::MAX_SPECIES) return "n_species must be in 1..4";
    if (d->precision != TURSCA_FP64 && d->precision != TURSCA_FP32_REFINE) return "unknown precision";
    if (d->coupling_mode != TURSCA_COUPLING_NONE && d->coupling_mode != TURSCA_COUPLING_WEIGHT)
        return "unknown coupling_mode";
    if (d->stencil_radius < 1 || d->stencil_radius > 2) return "stencil_radius must be 1 or 2";
    if (d->nx < 2 * d->stencil_radius + 1 || d->ny < 2 * d->stencil_radius + 1)
        return "nx and ny must be at least 2 * stencil_radius + 1";
    if (d->nz < d->stencil_radius) return "nz must be at least stencil_radius";
    if (!(d->hx > 0 && d->hy > 0 && d->hz > 0) || !std::isfinite(d->hx) || !std::isfinite(d->hy) ||
        !std::isfinite(d->hz))
        return "cell sizes must be positive and finite";
    if (d->fib_points < 64 || d->fib_points > (1 << 24)) return "fib_points must be in [64, 2^24]";
    if ((long long)d->nx * d->ny * (d->nz + 1) > 200000000LL) return "grid too large";
    return std::string();
}

tursca_status ensure_fields(tursca_scene *sc) {
    if (sc->fields_alloc) return TURSCA_OK;
    const size_t es = sc->es;
    const size_t na = (size_t)sc->d.nx * sc->d.ny * sc->d.nz;
    const size_t nn = na + (size_t)sc->d.nx * sc->d.ny;
    CK(dalloc(sc->allocs, sc->mu_a, na * es), "alloc mu_a");
    CK(dalloc(sc->allocs, sc->mu_s, na * es * sc->d.n_species), "alloc mu_s");
    CK(dalloc(sc->allocs, sc->mu_e, na * es), "alloc mu_e");
    CK(dalloc(sc->allocs, sc->mu_st, na * es), "alloc mu_st");
    CK(dalloc(sc->allocs, sc->tsun, nn * es), "alloc tsun");
    CK(dalloc(sc->allocs, sc->e1, nn * es), "alloc e1");
    {
        // haloed arrays of the edge kernel (zeroed once: halo-free entries of
        // the ground layer are never read but stay defined)
        const size_t H = (size_t)sc->d.stencil_radius;
        const size_t npd = (size_t)(sc->d.nz + 1) * (sc->d.nx + 2 * H) * (sc->d.ny + 2 * H);
        void **hal[6] = {(void **)&sc->zc_iso, (void **)&sc->zc_sun, &sc->rt_h, &sc->mu_e_h, &sc->e1_h, &sc->wsp_h};
        for (int k = 0; k < 6; ++k) {
            const size_t bytes = npd * es * (k == 5 ? (size_t)sc->d.n_species : 1);
            CK(dalloc(sc->allocs, *hal[k], bytes), "alloc haloed");
            CK(cudaMemsetAsync(*hal[k], 0, bytes, sc->st), "memset haloed");
        }
        CK(dalloc(sc->allocs, sc->mu_x, 4 * na * es), "alloc extended extinction");
        const size_t rbytes = npd * es * (size_t)tk::srec_stride(sc->d.n_species);
        CK(dalloc(sc->allocs, sc->srec, rbytes), "alloc haloed");
        CK(cudaMemsetAsync(sc->srec, 0, rbytes, sc->st), "memset haloed");
    }
    CK(dalloc(sc->allocs, sc->s, nn * es), "alloc s");
    CK(dalloc(sc->allocs, sc->gsun, na * es), "alloc gsun");
    CK(dalloc(sc->allocs, sc->emis, na * es), "alloc emis");
    CK(dalloc(sc->allocs, sc->musmax, sizeof(unsigned long long)), "alloc musmax");
    CK(dalloc(sc->allocs, sc->status, sizeof(int)), "alloc status");
    CK(cudaMemsetAsync(sc->status, 0, sizeof(int), sc->st), "memset status");
    // solver vectors live in the haloed layout (border of stencil_radius)
    const size_t H = (size_t)sc->d.stencil_radius;
    const size_t np = (size_t)(sc->d.nz + 1) * (sc->d.nx + 2 * H) * (sc->d.ny + 2 * H);
    CK(dalloc(sc->allocs, sc->x64, np * sizeof(double)), "alloc x");
    CK(dalloc(sc->allocs, sc->r64, np * sizeof(double)), "alloc r");
    // partial sums: the residual writes one per row block (4 per group of 128
    // rows), the power sweeps two columns of those, the dot products up to 64 x 296
    {
        const size_t groups = (size_t)(sc->d.nz + 1) * (((size_t)sc->d.nx * sc->d.ny + tk::kGroup - 1) / tk::kGroup);
        CK(dalloc(sc->allocs, sc->part, std::max<size_t>(64 * 1024, 8 * groups + 64) * sizeof(double)),
           "alloc part");
    }
    CK(dalloc(sc->allocs, sc->dred, 256 * sizeof(double)), "alloc red");
    CK(dalloc(sc->allocs, sc->b, np * es), "alloc b");
    CK(dalloc(sc->allocs, sc->d0, np * es), "alloc d0");
    CK(dalloc(sc->allocs, sc->d1, np * es), "alloc d1");
    CK(dalloc(sc->allocs, sc->w, np * es), "alloc w");
    CK(dalloc(sc->allocs, sc->xh, np * sizeof(float)), "alloc xh");
    CK(dalloc(sc->allocs, sc->xl, np * sizeof(float)), "alloc xl");
    if (!sc->hred) {
        cudaError_t e = cudaMallocHost((void **)&sc->hred, 256 * sizeof(double));
        if (e != cudaSuccess) return cuda_fail(sc, e, "alloc pinned");
    }
    sc->fields_alloc = true;
    return TURSCA_OK;
}

tursca_status sync_check(tursca_scene *sc, const char *where) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(sc->st);
    if (e != cudaSuccess) return cuda_fail(sc, e, where);
    if (sc->status) {
        int stv = 0;
        e = cudaMemcpy(&stv, sc->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(sc, e, where);
        if (stv & tk::STATUS_BAD_FIELD)
            return fail(sc, TURSCA_E_INVALID, "field values must be finite and non-negative");
        if (stv & tk::STATUS_TIMEOUT) return fail(sc, TURSCA_E_TIMEOUT, "a bounded device wait gave up");
    }
    return TURSCA_OK;
}

// ---------------------------------------------------------------------------
// Solver

struct SolveState {
    int iters = 0, refinements = 0, solver = 0;
    double rel = 1.0, rho = 0.0;
};

template <typename T>
tursca_status read_red(tursca_scene *sc, int n) {
    CK(cudaMemcpyAsync(sc->hred, sc->dred, n * sizeof(double), cudaMemcpyDeviceToHost, sc->st), "d2h");
    // the status word rides along: a bounded wait that gave up shows here
    int *hst = (int *)(sc->hred + 255);
    CK(cudaMemcpyAsync(hst, sc->status, sizeof(int), cudaMemcpyDeviceToHost, sc->st), "d2h");
    CK(cudaStreamSynchronize(sc->st), "sync");
    // invalid field values flagged by the assembly (the node-form solve
    // starts without waiting for it, so they are first seen here)
    if (*hst & tk::STATUS_BAD_FIELD) return fail(sc, TURSCA_E_INVALID, "field values must be finite and non-negative");
    if (*hst & tk::STATUS_TIMEOUT) return fail(sc, TURSCA_E_TIMEOUT, "a bounded device wait gave up");
    return TURSCA_OK;
}

// Neumann (source) iteration on (I - K) d = b: d <- b + K d, n sweeps after d = b.
template <typename T>
T *neumann(tursca_scene *sc, const tk::GridC &g, const tk::GraphP &gp, const T *val, const T *b, int n,
          SolveState &ss) {
    T *cur = (T *)sc->d0, *nxt = (T *)sc->d1;
    cudaMemcpyAsync(cur, b, (size_t)g.npad * sizeof(T), cudaMemcpyDeviceToDevice, sc->st);  // checked at the next sync
    for (int it = 0; it < n; ++it) {
        int pi = prof_begin(sc, P_SPMV);
        tk::launch_spmv<T>(sc->st, g, gp, val, cur, b, nxt);
        prof_end(sc, pi);
        std::swap(cur, nxt);
    }
    sc->launches += n;
    ss.iters += n;
    return cur;
}

// Restarted GMRES(m) on (I - K) d = b to ||b - (I - K) d|| <= tol ||b||; d must
// not alias b.  Classical Gram-Schmidt with one re-orthogonalisation pass.
template <typename T>
tursca_status gmres(tursca_scene *sc, const tk::GridC &g, const tk::GraphP &gp, const T *val, const T *b, T *d,
                    double tol, int maxit, SolveState &ss) {
    const int n = (int)g.npad, m = sc->gm_m;  // haloed vectors
    const size_t ld = (size_t)n;
    T *V = (T *)sc->V, *w = (T *)sc->w, *r = (T *)sc->d1;
    T *z0 = V + (size_t)(m + 1) * ld, *z1 = V + (size_t)(m + 2) * ld;  // preconditioner work vectors
    // dst = (I + K + ... + K^(kGmresPoly - 1)) src by Horner passes y = src + K y,
    // alternating between tmp and dst so that the last pass lands in dst
    auto apply_poly = [&](const T *src, T *dst, T *tmp) {
        const T *in = src;
        for (int p = 1; p < kGmresPoly; ++p) {
            T *out = ((kGmresPoly - 1 - p) % 2 == 0) ? dst : tmp;
            tk::launch_spmv<T>(sc->st, g, gp, val, in, src, out);
            in = out;
        }
        sc->launches += kGmresPoly - 1;
    };
    const int nb = tk::dot_blocks(g);
    CK(cudaMemsetAsync(d, 0, (size_t)n * sizeof(T), sc->st), "memset");
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
    tk::launch_sumsq<T>(sc->st, g, b, sc->part, nb, sc->dred);
    sc->launches += 2;
    tursca_status rs = read_red<T>(sc, 1);
    if (rs) return rs;
    const double bn = std::sqrt(sc->hred[0]);
    if (bn == 0.0) return TURSCA_OK;
    int total = 0;
    const T *rc = b;  // residual of the current cycle
    double beta = bn;
    for (int cycle = 0; cycle < 1000; ++cycle) {
        tk::launch_scale<T>(sc->st, n, rc, 1.0 / beta, V);
        sc->launches++;
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = beta;
        int k = 0;
        bool done = false;
        for (k = 0; k < m; ++k) {
            T *vk = V + (size_t)k * ld, *vn = V + (size_t)(k + 1) * ld;
            int pi = prof_begin(sc, P_GPROD);
            if (kGmresPoly > 1) {
                apply_poly(vk, z0, z1);  // z = M^-1 v_k
                tk::launch_imk<T>(sc->st, g, gp, val, z0, w);
            } else {
                tk::launch_imk<T>(sc->st, g, gp, val, vk, w);
            }
            prof_end(sc, pi, kGmresPoly);
            int po = prof_begin(sc, P_ORTH);
            tk::launch_dots<T, T>(sc->st, g, V, ld, k + 1, w, sc->part, nb, sc->dred);
            tk::launch_gmres_update<T>(sc->st, n, w, V, ld, k + 1, sc->dred);
            tk::launch_dots<T, T>(sc->st, g, V, ld, k + 1, w, sc->part, nb, sc->dred + 64);
            tk::launch_gmres_update_norm<T>(sc->st, g, n, w, V, ld, k + 1, sc->dred + 64, sc->part, nb, sc->dred + 128);
            prof_end(sc, po);
            sc->launches += 9;
            ss.iters++;
            total++;
            CK(cudaMemcpyAsync(sc->hred, sc->dred, 129 * sizeof(double), cudaMemcpyDeviceToHost, sc->st), "d2h");
            CK(cudaStreamSynchronize(sc->st), "sync");
            for (int i = 0; i <= k; ++i) H[(size_t)i * m + k] = sc->hred[i] + sc->hred[64 + i];
            double hn = std::sqrt(std::max(0.0, sc->hred[128]));
            H[(size_t)(k + 1) * m + k] = hn;
            if (hn > 0.0) {
                tk::launch_scale<T>(sc->st, n, w, 1.0 / hn, vn);
                sc->launches++;
            }
            for (int i = 0; i < k; ++i) {
                double a = H[(size_t)i * m + k], c = H[(size_t)(i + 1) * m + k];
                H[(size_t)i * m + k] = cs[i] * a + sn[i] * c;
                H[(size_t)(i + 1) * m + k] = -sn[i] * a + cs[i] * c;
            }
            double a = H[(size_t)k * m + k], c = H[(size_t)(k + 1) * m + k];
            double den = std::sqrt(a * a + c * c);
            cs[k] = den > 0 ? a / den : 1.0;
            sn[k] = den > 0 ? c / den : 0.0;
            H[(size_t)k * m + k] = den;
            H[(size_t)(k + 1) * m + k] = 0.0;
            gv[k + 1] = -sn[k] * gv[k];
            gv[k] = cs[k] * gv[k];
            if (std::fabs(gv[k + 1]) <= tol * bn || hn == 0.0 || total >= maxit) {
                ++k;
                done = true;
                break;
            }
        }
        if (k > m) k = m;
        for (int i = k - 1; i >= 0; --i) {
            double acc = gv[i];
            for (int j = i + 1; j < k; ++j) acc -= H[(size_t)i * m + j] * y[j];
            y[i] = H[(size_t)i * m + i] != 0.0 ? acc / H[(size_t)i * m + i] : 0.0;
        }
        CK(cudaMemcpyAsync(sc->dred + 192, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, sc->st), "h2d");
        if (kGmresPoly > 1) {
            // d += M^-1 (V y)
            CK(cudaMemsetAsync(z0, 0, (size_t)n * sizeof(T), sc->st), "memset");
            tk::launch_combine<T>(sc->st, n, z0, V, ld, k, sc->dred + 192);
            apply_poly(z0, w, z1);
            tk::launch_add<T>(sc->st, n, d, w);
            sc->launches += 3;
        } else {
            tk::launch_combine<T>(sc->st, n, d, V, ld, k, sc->dred + 192);
            sc->launches++;
        }
        // true residual r = b - (I - K) d
        tk::launch_imk<T>(sc->st, g, gp, val, d, w);
        tk::launch_axpby<T>(sc->st, n, 1.0, b, -1.0, w, r);
        tk::launch_sumsq<T>(sc->st, g, r, sc->part, nb, sc->dred);
        sc->launches += 4;
        ss.iters++;
        rs = read_red<T>(sc, 1);
        if (rs) return rs;
        double nb_ = std::sqrt(sc->hred[0]);
        if (nb_ <= tol * bn * 1.0000001 || total >= maxit || nb_ == 0.0) break;
        if (!(nb_ < 0.5 * beta)) break;  // the cycle stagnated (rounding floor)
        beta = nb_;
        rc = r;
        (void)done;
    }
    return TURSCA_OK;
}

// The solve's schedule constants: the power sweeps of the first refinement
// and the lower end of the Chebyshev interval as a fraction of its upper end.
// Chosen on a model of this loop (float32 K from an FP64 reference, the same
// planning rules) over plume scenes of 16^3 to 64^2 x 32 voxels, SZA 20 to 75
// degrees, and random scenes: 4 sweeps and -0.4 b take 3 refinements in every
// case and about 5% less solve time than 6 sweeps and -0.5 b; on the 64^2 x 32
// plume, 4 sweeps + 30 Chebyshev steps against 6 + 30.  The plume's spectrum
// lies in [-0.229, 0.610] (ARPACK), inside [-0.4 b, b] for b = 1.02 x the
// power estimate (0.67) + 0.005.
#ifndef TK_POWER_SWEEPS
#define TK_POWER_SWEEPS 4
#endif
#ifndef TK_CHEB_LO
#define TK_CHEB_LO 0.4
#endif

// Chebyshev iteration parameters for A = I - K with the eigenvalues of K taken
// in [lo, hi] (real, hi < 1): A's eigenvalues lie in [1 - hi, 1 - lo].
struct ChebPlan {
    double theta, delta, sigma, rate;
};
ChebPlan cheb_plan(double lo, double hi) {
    ChebPlan c;
    double alpha = 1.0 - hi, beta = 1.0 - lo;
    c.theta = 0.5 * (alpha + beta);
    c.delta = 0.5 * (beta - alpha);
    c.sigma = c.theta / c.delta;
    c.rate = 1.0 / (c.sigma + std::sqrt(c.sigma * c.sigma - 1.0));  // asymptotic error factor per step
    return c;
}

// What a solve works on: K (graph and values) or K^T (the transposed ones),
// the source (node order) and the FP64 solution (haloed).
template <typename T>
struct SolveIO {
    tk::GridC g;
    tk::GraphP gp;
    const T *val;
    const T *s;
    double *x;
};

template <typename T>
SolveIO<T> forward_io(tursca_scene *sc) {
    SolveIO<T> io;
    io.g = grid_c(sc);
    io.gp = graph_p(sc);
    io.val = (const T *)sc->val;
    io.s = (const T *)sc->s;
    io.x = sc->x64;
    return io;
}

// The values of K in the persisting part of L2 for the passes of one solve
// (TURSCA_OPT_L2_RESIDENT): every pass of a solve streams the same values,
// and a scene's values often fit in the 126 MB L2.  The window covers the
// values (the fraction of it that the set-aside holds, by address); when the
// solve ends the window is removed and the persisting lines return to normal
// status, so later work finds an ordinary cache.
struct L2Window {
    cudaStream_t st = nullptr;
    L2Window(tursca_scene *sc, const void *base, size_t bytes) {
        if (!sc->l2_resident || !base || !bytes) return;
        int dev = 0, maxw = 0;
        size_t lim = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, dev);
        cudaDeviceGetLimit(&lim, cudaLimitPersistingL2CacheSize);
        if (maxw <= 0 || lim == 0) return;
        cudaStreamAttrValue a = {};
        a.accessPolicyWindow.base_ptr = const_cast<void *>(base);
        a.accessPolicyWindow.num_bytes = std::min(bytes, (size_t)maxw);
        a.accessPolicyWindow.hitRatio = (float)std::min(1.0, (double)lim / (double)a.accessPolicyWindow.num_bytes);
        a.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        a.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        if (cudaStreamSetAttribute(sc->st, cudaStreamAttributeAccessPolicyWindow, &a) == cudaSuccess) st = sc->st;
    }
    ~L2Window() {
        if (!st) return;
        cudaStreamAttrValue a = {};
        a.accessPolicyWindow.num_bytes = 0;
        cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &a);
        cudaStreamSynchronize(st);
        cudaCtxResetPersistingL2Cache();
    }
};

template <typename T>
tursca_status do_solve(tursca_scene *sc, int solver, double rtol, int max_iter, tursca_solve_info *info,
                       const SolveIO<T> &io) {
    const L2Window l2w(sc, io.val, (size_t)sc->G.nval * sizeof(T));
    const tk::GridC &g = io.g;
    const tk::GraphP &gp = io.gp;
    const T *val = io.val;
    const int n = (int)g.npad;  // solver vectors are haloed
    const int nbr = tk::resid_blocks(g);
    const int nb = tk::dot_blocks(g);
    const int nsw = tk::sweep_blocks(g);
    SolveState ss;
    (void)nb;
    const bool fp64 = sc->d.precision == TURSCA_FP64;
    if (solver == TURSCA_SOLVER_AUTO) solver = fp64 ? TURSCA_SOLVER_GMRES : TURSCA_SOLVER_CHEBYSHEV;
    auto ensure_basis = [&]() -> tursca_status {
        int m = fp64 ? 40 : TK_GMRES_M32;
        if (!sc->V || sc->gm_m != m) {
            T *V;
            // m + 1 basis vectors and two work vectors of the preconditioner
            CK(dalloc(sc->allocs, V, (size_t)(m + 3) * n * sizeof(T)), "alloc gmres basis");
            sc->V = V;
            sc->gm_m = m;
        }
        return TURSCA_OK;
    };
    // residual arithmetic: FP32 pairs on FP32 scenes (FP64 runs at a small
    // fraction of the FP32 rate on this GPU), FP64 on FP64 scenes or on request
    const bool ds = !fp64 && !sc->resid_fp64 && tk::resid_ds_ok(g);
    // x = 0, r = s, ||s||
    CK(cudaMemsetAsync(io.x, 0, (size_t)n * sizeof(double), sc->st), "memset x");
    tk::launch_to_halo<T, double>(sc->st, g, io.s, sc->r64);
    // ||s||^2 goes to dred[4] and is read with the first refinement's residual
    tk::launch_sumsq<double>(sc->st, g, sc->r64, sc->part, nb, sc->dred + 4);
    sc->launches += 3;
    tursca_status rs = TURSCA_OK;
    double sn = -1.0;  // not read yet
    double rel = 1.0;
    double rho = -1.0;      // estimate of the largest eigenvalue of K (-1: none yet)
    double widen = 0.0;     // extra margin after a refinement that under-delivered
    int inner_n = 8;        // Neumann sweeps (explicit Neumann solver)
    int stalls = 0;
    bool use_gmres = false;       // Chebyshev under-delivered: GMRES from now on
    const double floor32 = 3e-7;  // relative accuracy the FP32 inner iterations can reach
    while (rel > rtol && ss.iters < max_iter) {
        const int budget = max_iter - ss.iters;
        T *bb = (T *)sc->b;  // r in the compute type (written below, with the first pass of each solver)
        // reduction asked of this refinement: all that is left if one
        // refinement can reach it, else an equal share over the fewest
        // refinements the FP32 floor allows
        const double need = rtol / rel;
        double target;
        if (fp64 || need >= 10.0 * floor32) {
            target = std::max(0.3 * need, fp64 ? 1e-15 : floor32);
        } else {
            int m = (int)std::ceil(std::log(need) / std::log(10.0 * floor32));
            target = 0.3 * std::max(std::pow(need, 1.0 / m), 10.0 * floor32);
        }
        const T *dd = nullptr;
        bool x_done = false;  // x += dd already applied by the last pass of the inner solve
        int kind = solver;
        bool power = false;
        double predicted = 1.0;
        if (solver == TURSCA_SOLVER_CHEBYSHEV) {
            // Chebyshev on a real interval needs a clear gap below 1: near 1 the
            // (small) imaginary parts of the spectrum in the middle of the
            // interval are amplified, so GMRES takes over there
            if (rho < 0.0)
                power = true;
            else if (rho + widen >= 0.85 || use_gmres)
                kind = TURSCA_SOLVER_GMRES;
        }
        if (power || kind != TURSCA_SOLVER_CHEBYSHEV) {
            tk::launch_convert<double, T>(sc->st, n, sc->r64, bb);
            sc->launches++;
        }
        if (power) {
            // Neumann sweeps d <- r + K d from d = r; the norms of successive
            // differences (K^k r) give the power estimate of the largest eigenvalue
            const int n1 = std::max(2, std::min(TK_POWER_SWEEPS, budget - 1));
            // the first sweep reads d = r from bb itself; the later ones
            // alternate between d0 and d1, so bb is never overwritten
            T *cur = bb, *nxt = (T *)sc->d0;
            int pi = prof_begin(sc, P_SPMV);
            for (int it = 0; it < n1; ++it) {
                // the last sweep also applies x += d (its output) row by row
                const bool last = it == n1 - 1;
                tk::launch_sweep_pow<T>(sc->st, g, gp, val, cur, bb, nxt, sc->part + (it & 1) * nsw,
                                        last ? io.x : nullptr, last && ds ? sc->xh : nullptr,
                                        last && ds ? sc->xl : nullptr);
                
                cur = nxt;
                nxt = cur == (T *)sc->d0 ? (T *)sc->d1 : (T *)sc->d0;
            }
            prof_end(sc, pi, n1);
            tk::launch_finalize2(sc->st, sc->part, nsw, sc->dred + 2);
            sc->launches += n1 + 1;
            ss.iters += n1;
            dd = cur;
            x_done = true;
            ss.solver = TURSCA_SOLVER_NEUMANN;
            // columns: last sweep (n1 - 1) & 1, the one before (n1 - 2) & 1
            inner_n = n1;
        } else if (kind == TURSCA_SOLVER_CHEBYSHEV) {
            const double hi = std::min(0.9995, 1.02 * (rho + widen) + 0.005);
            const ChebPlan cp = cheb_plan(-TK_CHEB_LO * hi, hi);
            // K is not normal: the error contracts more slowly than the
            // interval bound says (measured ~ rate^0.65 per step on the plume)
            const double eff = std::pow(cp.rate, 0.65);
            int nc = (int)std::ceil(std::log(target / 2.0) / std::log(eff));
            nc = std::max(1, std::min(nc, budget - 1));
            predicted = 2.0 * std::pow(eff, nc);
            T *r = bb, *d = (T *)sc->w, *p0 = (T *)sc->d0, *p1 = (T *)sc->d1;
            tk::launch_cheb_start<T>(sc->st, n, sc->r64, 1.0 / cp.theta, r, d, p0);
            sc->launches++;
            // in a server: hand the refinement to the batcher, which runs it
            // in one persistent launch with the refinements of other requests
            bool batched = false;
            if constexpr (sizeof(T) == 4) {
                if (sc->batcher && tk::batch_eligible(g, nc)) {
                    tk::ChebJob job;
                    std::memset(&job, 0, sizeof(job));
                    job.g = g;
                    job.gp = gp;
                    job.val = (const float *)val;
                    job.r = (float *)r;
                    job.d = (float *)d;
                    job.p[0] = (float *)p0;
                    job.p[1] = (float *)p1;
                    job.x64 = io.x;
                    job.xh = ds ? sc->xh : nullptr;
                    job.xl = ds ? sc->xl : nullptr;
                    job.nsteps = nc;
                    job.W = g.wq;
                    double rk = 1.0 / cp.sigma;
                    for (int k = 0; k < nc; ++k) {  // the coefficients the scene's own passes would take
                        const double rk1 = 1.0 / (2.0 * cp.sigma - rk);
                        job.c1[k] = (float)(rk1 * rk);
                        job.c2[k] = (float)(2.0 * rk1 / cp.delta);
                        rk = rk1;
                    }
                    CK(cudaEventRecord(sc->bready, sc->st), "batch event");
                    if (tk::batcher_run(sc->batcher, job, sc->bready, sc->bdone)) {
                        CK(cudaStreamWaitEvent(sc->st, sc->bdone, 0), "batch wait");
                        batched = true;
                    }
                }
            }
            if (!batched) {
                double rk = 1.0 / cp.sigma;
                int pi = prof_begin(sc, P_CHEB);
                for (int k = 0; k < nc; ++k) {
                    double rk1 = 1.0 / (2.0 * cp.sigma - rk);
                    // the last step also applies x += d row by row
                    const bool last = k == nc - 1;
                    tk::launch_cheb<T>(sc->st, g, gp, val, p0, r, d, p1, rk1 * rk, 2.0 * rk1 / cp.delta,
                                       last ? io.x : nullptr, last && ds ? sc->xh : nullptr,
                                       last && ds ? sc->xl : nullptr);
                    std::swap(p0, p1);
                    rk = rk1;
                }
                prof_end(sc, pi, nc);
                sc->launches += nc;
            }
            ss.iters += nc;
            dd = d;
            x_done = true;
            ss.solver = TURSCA_SOLVER_CHEBYSHEV;
        } else if (kind == TURSCA_SOLVER_GMRES) {
            tursca_status e = ensure_basis();
            if (e) return e;
            if (sn < 0.0) {  // GMRES reuses the reduction buffer: read ||s|| first
                rs = read_red<T>(sc, 5);
                if (rs) return rs;
                sn = std::sqrt(sc->hred[4]);
            }
            double tol = fp64 ? std::max(0.3 * rtol / rel, 1e-15) : std::max(0.3 * rtol / rel, 2e-6);
            e = gmres<T>(sc, g, gp, val, bb, (T *)sc->d0, tol, budget, ss);
            if (e) return e;
            dd = (const T *)sc->d0;
            ss.solver = TURSCA_SOLVER_GMRES;
        } else {  // Neumann
            int nn = std::min(inner_n, std::max(1, budget - 1));
            dd = neumann<T>(sc, g, gp, val, bb, nn, ss);
            inner_n = nn;
            ss.solver = TURSCA_SOLVER_NEUMANN;
        }
        if (!x_done) tk::launch_update_x<T>(sc->st, n, dd, io.x, ds ? sc->xh : nullptr, ds ? sc->xl : nullptr);
        int pr = prof_begin(sc, P_RESID);
        if (ds)
            tk::launch_resid_ds(sc->st, g, gp, (const float *)val, (const float *)io.s, io.x, sc->xh, sc->xl,
                                sc->r64, sc->part, nbr);
        else
            tk::launch_resid64<T>(sc->st, g, gp, val, io.s, io.x, sc->r64, sc->part,
                                  nbr);
        prof_end(sc, pr);
        tk::launch_finalize(sc->st, sc->part, nbr, sc->dred);
        sc->launches += 3;
        ss.refinements++;
        ss.iters++;
        rs = read_red<T>(sc, 5);
        if (rs) return rs;
        if (sn < 0.0) sn = std::sqrt(sc->hred[4]);
        const double prev = rel;
        rel = sn > 0 ? std::sqrt(sc->hred[0]) / sn : 0.0;
        const double f = prev > 0 ? rel / prev : 0.0;
        if (power) {
            const int n1 = inner_n;
            double last = sc->hred[2 + ((n1 - 1) & 1)], before = sc->hred[2 + ((n1 - 2) & 1)];
            double est = before > 0 ? std::sqrt(last / before) : 0.0;
            // the series' own reduction bounds the estimate from below
            double avg = (f > 0 && f < 1) ? std::pow(f, 1.0 / (n1 + 1)) : 0.0;
            rho = std::min(0.9999, std::max(est, avg));
            ss.rho = rho;
        } else if (kind == TURSCA_SOLVER_CHEBYSHEV) {
            if (f > std::max(30.0 * predicted, 3.0 * floor32) && rel > rtol) {
                // the interval missed part of the spectrum: widen it once toward 1,
                // or hand over to GMRES
                if (f > 0.5 || widen > 0.0 || rho + 0.5 * (1.0 - rho) > 0.95)
                    use_gmres = true;
                else
                    widen += 0.5 * (1.0 - (rho + widen));
                ++stalls;
            }
        } else if (kind == TURSCA_SOLVER_NEUMANN && solver == TURSCA_SOLVER_NEUMANN) {
            if (prev > 0 && rel > 0 && f < 1.0) {
                double rr = std::pow(std::min(f, 0.999999), 1.0 / (inner_n + 1));
                if (ss.refinements == 1 || f > 1e-6) ss.rho = rr;
                double tg = fp64 ? std::max(rtol / rel * 0.3, 1e-15) : std::max(rtol / rel * 0.3, 1e-6);
                int want = (int)std::ceil(std::log(tg) / std::log(std::max(ss.rho, 1e-3))) - 1;
                inner_n = std::max(2, std::min(want, 400));
            }
        }
        if (!(rel <= prev * 1.5) && ss.refinements > 3) break;  // diverging
        if (stalls > 6) break;
    }
    if (info) {
        info->iters = ss.iters;
        info->refinements = ss.refinements;
        info->rel_resid64 = rel;
        info->rho_est = ss.rho;
        info->solver = ss.solver;
    }
    sc->solved = true;
    if (rel > rtol) return fail(sc, TURSCA_E_NOT_CONVERGED, "solver stopped above rtol");
    return TURSCA_OK;
}

template <typename T>
tursca_status do_render(tursca_scene *sc, void *radiance, void *reflectance) {
    const tk::GridC g = grid_c(sc);
    const tk::GraphP gp = graph_p(sc);
    tk::FieldP<T> f = field_p<T>(sc);
    tk::ViewC vc = view_c(sc);
    tk::ViewP vp = view_p(sc);
    int pi = prof_begin(sc, P_RENDER);
    if (sc->aniso_asm) {
        // the emission came with the solve (from X)
    } else if (sc->single_asm) {
        tk::launch_emission_first<T>(sc->st, g, f, (T *)sc->emis);
    } else {
        // the solution in the compute type, gathered by the emission kernel
        const T *xc;
        if constexpr (sizeof(T) == 8) {
            xc = (const T *)sc->x64;
        } else {
            tk::launch_convert<double, T>(sc->st, (int)g.npad, sc->x64, (T *)sc->w);
            sc->launches++;
            xc = (const T *)sc->w;
        }
        tk::launch_emission<T>(sc->st, g, gp, f, vc, xc, (T *)sc->emis);
    }
    tk::launch_pixels<T>(sc->st, g, f, vc, vp, (const T *)sc->emis, sc->x64, (T *)sc->rad, (T *)sc->refl);
    prof_end(sc, pi);
    sc->launches += 2;
    size_t np = (size_t)sc->geom.npx * sc->geom.npy;
    CK(cudaGetLastError(), "render launch");
    if (radiance) CK(cudaMemcpyAsync(radiance, sc->rad, np * sizeof(T), cudaMemcpyDefault, sc->st), "copy radiance");
    if (reflectance)
        CK(cudaMemcpyAsync(reflectance, sc->refl, np * sizeof(T), cudaMemcpyDefault, sc->st), "copy reflectance");
    tursca_status rs = sync_check(sc, "render");
    sc->rendered = rs == TURSCA_OK;
    return rs;
}

// ---------------------------------------------------------------------------
// Adjoint

tursca_status ensure_adjoint(tursca_scene *sc) {
    if (sc->adj_ready) return TURSCA_OK;
    const tg::Graph &G = sc->G;
    const tk::GridC g = grid_c(sc);
    tg::Transposed Tt;
    tg::transpose_templates(G, g.H, Tt);
    const size_t ne = Tt.recv_layer.size();
    std::vector<int4> info(ne);
    std::vector<int> hg(ne);
    for (size_t e = 0; e < ne; ++e) {
        const int i = Tt.tmpl_index[e], zi = Tt.recv_layer[e];
        const tg::TSlot &t = G.tmpl[i];
        info[e] = make_int4(i - G.tmpl_start[zi], zi, t.sdx, t.sdy);
        hg[e] = G.classes[t.cls].hgdir;
    }
    if (Tt.voff[g.nz + 1] != G.nval) return fail(sc, TURSCA_E_INVALID, "internal error: K^T size");
    CK(upload(sc, sc->allocs, sc->tstartT, Tt.tstart.data(), Tt.tstart.size() * sizeof(int)), "upload K^T");
    CK(upload(sc, sc->allocs, sc->voffT, Tt.voff.data(), Tt.voff.size() * sizeof(long long)), "upload K^T");
    CK(upload(sc, sc->allocs, sc->infoT, info.data(), std::max<size_t>(1, ne) * sizeof(int4)), "upload K^T");
    CK(upload(sc, sc->allocs, sc->flatT, Tt.flat_h.data(), std::max<size_t>(1, ne) * sizeof(int)), "upload K^T");
    CK(upload(sc, sc->allocs, sc->hgdirT, hg.data(), std::max<size_t>(1, ne) * sizeof(int)), "upload K^T");
    {
        tg::TileLayout tl;
        sc->tile_tlT = 0;
        if (ne && tg::tile_layout(G, Tt, g.H, tl).empty() &&
            (size_t)tk::kTileLayers * tl.tl * sizeof(float) <= (size_t)tk::kTileMaxBytes) {
            CK(upload(sc, sc->allocs, sc->ttileT, tl.ttile.data(), tl.ttile.size() * sizeof(int)), "upload K^T tiles");
            CK(upload(sc, sc->allocs, sc->tlayT, tl.layers.data(), tl.layers.size() * sizeof(int)), "upload K^T tiles");
            sc->tile_tlT = tl.tl;
        }
    }
    const size_t es = sc->es;
    CK(dalloc(sc->allocs, sc->valT, (size_t)G.nval * es), "alloc K^T");
    CK(dalloc(sc->allocs, sc->lam64, (size_t)g.npad * sizeof(double)), "alloc adjoint");
    CK(dalloc(sc->allocs, sc->Lbar, (size_t)sc->geom.npx * sc->geom.npy * es), "alloc adjoint");
    const size_t nn = (size_t)g.n_nodes, na = (size_t)g.n_atm, np = (size_t)g.npad;
    const size_t sz[10] = {nn, np, nn, np, nn, na, np, (size_t)g.nc * np, (size_t)g.nup * na, (size_t)g.ngd * g.lp};
    for (int k = 0; k < 10; ++k) {
        sc->adj_bytes[k] = std::max<size_t>(1, sz[k]) * es;
        CK(dalloc(sc->allocs, sc->adj[k], sc->adj_bytes[k]), "alloc adjoint");
    }
    CK(cudaStreamSynchronize(sc->st), "sync");
    sc->adj_ready = true;
    return TURSCA_OK;
}

template <typename T>
tursca_status do_adjoint(tursca_scene *sc, const void *dJ_dL, void *dJ_dmu_abs) {
    tk::GridC g = grid_c(sc);
    const tk::GraphP gp = graph_p(sc);
    tk::FieldP<T> f = field_p<T>(sc);
    const tk::ViewC vc = view_c(sc);
    const tk::ViewP vp = view_p(sc);
    tk::TransP tp;
    tp.tstart = sc->tstartT;
    tp.voff = sc->voffT;
    tp.info = sc->infoT;
    tp.flat = sc->flatT;
    tp.hgdir = sc->hgdirT;
    tk::GraphP gpT = gp;  // K^T: the same kind of templates over source layers
    gpT.tstart = sc->tstartT;
    gpT.voff = sc->voffT;
    gpT.tflat = sc->flatT;
    gpT.ttile = sc->ttileT;  // gather tiles of the K^T templates
    gpT.tlay = sc->tlayT;
    tk::AdjP<T> ad;
    T **slot[10] = {&ad.Ebar, &ad.Ebar_h, &ad.e1bar, &ad.e1bar_h, &ad.xbar,
                    &ad.mubar, &ad.mubar_h, &ad.tsegbar, &ad.tinfbar, &ad.tinfgbar};
    for (int k = 0; k < 10; ++k) {
        *slot[k] = (T *)sc->adj[k];
        CK(cudaMemsetAsync(sc->adj[k], 0, sc->adj_bytes[k], sc->st), "memset adjoint");
    }
    const size_t npix = (size_t)sc->geom.npx * sc->geom.npy;
    CK(cudaMemcpyAsync(sc->Lbar, dJ_dL, npix * sizeof(T), cudaMemcpyDefault, sc->st), "copy dJ/dL");
    // K^T first: the launches after it are plain ones until the row-group passes
    tk::launch_transpose_vals<T>(sc->st, g, gp, tp, (const T *)sc->val, (T *)sc->valT);
    tk::launch_pix_adj<T>(sc->st, g, f, vc, vp, (const T *)sc->emis, sc->x64, (const T *)sc->Lbar, ad);
    tk::launch_to_halo<T, T>(sc->st, g, ad.Ebar, ad.Ebar_h);
    tk::launch_emis_adj<T>(sc->st, g, gpT, tp, f, (const T *)sc->valT, ad);
    sc->launches += 4;
    // (I - K)^T lambda = x-bar
    SolveIO<T> io;
    g.stage = 0;
    g.tl = sc->gather_tile ? sc->tile_tlT : 0;
    io.g = g;
    io.gp = gpT;
    io.val = (const T *)sc->valT;
    io.s = ad.xbar;
    io.x = sc->lam64;
    tursca_solve_info info;
    const double rtol = sc->d.precision == TURSCA_FP64 ? 1e-12 : 1e-9;
    tursca_status rs = do_solve<T>(sc, TURSCA_SOLVER_AUTO, rtol, 5000, &info, io);
    if (rs) return rs;
    if (sc->sel_asm)
        tk::launch_asm_adj_sel<T>(sc->st, grid_c(sc), gp, f, vc, sc->x64, sc->lam64, ad, (const T *)sc->w_iso,
                                  (const T *)sc->w_sun);
    else
        tk::launch_asm_adj<T>(sc->st, grid_c(sc), gp, f, vc, sc->x64, sc->lam64, ad);
    tk::launch_tables_adj<T>(sc->st, grid_c(sc), gp, f, vc, vp, ad);
    sc->launches += 6;
    CK(cudaGetLastError(), "adjoint launch");
    CK(cudaMemcpyAsync(dJ_dmu_abs, ad.mubar, (size_t)g.n_atm * sizeof(T), cudaMemcpyDefault, sc->st), "copy gradient");
    return sync_check(sc, "adjoint");
}

}  // namespace

// ===========================================================================
// C ABI

// Coupling selection: rank the directions by decreasing cosine to every
// lattice point (exact ties to the lower index, as in the partition), order
// the points of every cell by their rankings (so the points that a dropped
// cell hands to one kept direction sit together), do the same for the
// upper-hemisphere points and the ground cells, and allocate the per-scene
// buffers and the weight planes.  Once per scene.
tursca_status ensure_select(tursca_scene *sc) {
    if (sc->sel_ready) return TURSCA_OK;
    const tg::Graph &G = sc->G;
    const int M = G.M, nd = (int)G.dirs.size(), ngd = (int)G.gdirs.size();
    if (M > (1 << 20) || nd > tk::kSelMaxDir || ngd > tk::kSelMaxDir)
        return fail(sc, TURSCA_E_UNSUPPORTED, "coupling selection needs at most 2^20 lattice points");
    auto ranked = [](const std::array<double, 3> &s, const std::vector<std::array<double, 3>> &uh,
                     unsigned char *out) {
        const int n = (int)uh.size();
        std::vector<std::pair<double, int>> c(n);
        for (int u = 0; u < n; ++u) c[u] = {-(uh[u][0] * s[0] + uh[u][1] * s[1] + uh[u][2] * s[2]), u};
        std::sort(c.begin(), c.end());
        for (int u = 0; u < n; ++u) out[u] = (unsigned char)c[u].second;
    };
    // points of each cell, ordered by their rankings; rows in that order
    auto order_cells = [](const std::vector<unsigned char> &rk, int n, const std::vector<int> &start,
                          std::vector<int> &pts) {
        for (size_t c = 0; c + 1 < start.size(); ++c)
            std::sort(pts.begin() + start[c], pts.begin() + start[c + 1], [&](int a, int b) {
                return std::memcmp(&rk[(size_t)a * n], &rk[(size_t)b * n], n) < 0;
            });
    };
    std::vector<unsigned char> rk((size_t)M * nd);
    for (int m = 0; m < M; ++m) {
        ranked(G.lattice[m], G.uhat, &rk[(size_t)m * nd]);
        if (rk[(size_t)m * nd] != G.cell[m]) return fail(sc, TURSCA_E_INVALID, "lattice ranking");
    }
    std::vector<int> pts(G.cell_order.begin(), G.cell_order.end());
    order_cells(rk, nd, G.cell_start, pts);
    std::vector<unsigned char> rank((size_t)M * nd);
    std::vector<double> lat((size_t)3 * M);
    for (int p = 0; p < M; ++p) {
        std::memcpy(&rank[(size_t)p * nd], &rk[(size_t)pts[p] * nd], nd);
        for (int a = 0; a < 3; ++a) lat[(size_t)3 * p + a] = G.lattice[pts[p]][a];
    }
    std::vector<std::array<double, 3>> gh(ngd);
    for (int k = 0; k < ngd; ++k) gh[k] = G.gdirs[k].uhat;
    std::vector<int> upts;
    std::vector<double> gzsum(ngd, 0.0);
    double gztot = 0.0;
    std::vector<unsigned char> grk;
    for (int m = 0; m < M; ++m) {
        const auto &pt = G.lattice[m];
        if (!(pt[2] > 0.0)) continue;
        const size_t i = upts.size();
        upts.push_back(m);
        grk.resize((i + 1) * ngd);
        ranked(pt, gh, &grk[i * ngd]);
        gzsum[grk[i * ngd]] += pt[2];
        gztot += pt[2];
    }
    const int nup = (int)upts.size();
    std::vector<int> gstart(ngd + 1, 0);
    for (int i = 0; i < nup; ++i) gstart[grk[(size_t)i * ngd] + 1]++;
    for (int k = 0; k < ngd; ++k) gstart[k + 1] += gstart[k];
    std::vector<int> fill(gstart.begin(), gstart.end() - 1), gpts(nup);
    for (int i = 0; i < nup; ++i) gpts[fill[grk[(size_t)i * ngd]]++] = i;
    order_cells(grk, ngd, gstart, gpts);
    std::vector<unsigned char> grank((size_t)std::max(nup, 1) * std::max(ngd, 1));
    std::vector<double> gz(std::max(nup, 1)), glat((size_t)3 * std::max(nup, 1));
    for (int p = 0; p < nup; ++p) {
        std::memcpy(&grank[(size_t)p * ngd], &grk[(size_t)gpts[p] * ngd], ngd);
        gz[p] = G.lattice[upts[gpts[p]]][2];
        for (int a = 0; a < 3; ++a) glat[(size_t)3 * p + a] = G.lattice[upts[gpts[p]]][a];
    }
    // FP32 copies for the cosine search over short kept lists
    auto to_f4 = [](const std::vector<double> &v3) {
        std::vector<float4> f(std::max<size_t>(1, v3.size() / 3));
        for (size_t i = 0; i < v3.size() / 3; ++i)
            f[i] = make_float4((float)v3[3 * i], (float)v3[3 * i + 1], (float)v3[3 * i + 2], 0.f);
        return f;
    };
    std::vector<double> dh;
    for (int u = 0; u < nd; ++u) dh.insert(dh.end(), G.uhat[u].begin(), G.uhat[u].end());
    for (int k = 0; k < ngd; ++k) dh.insert(dh.end(), gh[k].begin(), gh[k].end());
    const std::vector<float4> latf = to_f4(lat), glatf = to_f4(glat), dirf = to_f4(dh);
    tk::SelP &q = sc->selp;
    unsigned char *d_rank = nullptr, *d_grank = nullptr;
    int *d_gstart = nullptr;
    double *d_gz = nullptr, *d_gzsum = nullptr, *d_lat = nullptr, *d_glat = nullptr;
    float4 *d_latf = nullptr, *d_glatf = nullptr, *d_dirf = nullptr;
    CK(upload(sc, sc->allocs, d_glat, glat.data(), glat.size() * sizeof(double)), "upload rank");
    CK(upload(sc, sc->allocs, d_latf, latf.data(), latf.size() * sizeof(float4)), "upload rank");
    CK(upload(sc, sc->allocs, d_glatf, glatf.data(), glatf.size() * sizeof(float4)), "upload rank");
    CK(upload(sc, sc->allocs, d_dirf, dirf.data(), dirf.size() * sizeof(float4)), "upload rank");
    CK(upload(sc, sc->allocs, d_rank, rank.data(), rank.size()), "upload rank");
    CK(upload(sc, sc->allocs, d_lat, lat.data(), lat.size() * sizeof(double)), "upload rank");
    CK(upload(sc, sc->allocs, d_grank, grank.data(), grank.size()), "upload rank");
    CK(upload(sc, sc->allocs, d_gstart, gstart.data(), gstart.size() * sizeof(int)), "upload ground cells");
    CK(upload(sc, sc->allocs, d_gz, gz.data(), gz.size() * sizeof(double)), "upload ground cells");
    CK(upload(sc, sc->allocs, d_gzsum, gzsum.data(), gzsum.size() * sizeof(double)), "upload ground cells");
    // HG per lattice point in FP64, then its copy, the cell sums and the
    // species totals in the compute type
    CK(dalloc(sc->allocs, q.hgpt,
              ((size_t)sc->d.n_species * M * 2 + (size_t)sc->d.n_species * (nd + 1)) * sizeof(double)),
       "alloc select");
    CK(dalloc(sc->allocs, q.musmax_bits, sizeof(unsigned long long)), "alloc select");
    q.dmax = std::max(nd, ngd);
    {
        const size_t nn = (size_t)sc->G.n_nodes;
        int ht = 1;
        while ((size_t)ht < 2 * nn) ht <<= 1;
        q.ht = ht;
        CK(dalloc(sc->allocs, q.mask, nn * sizeof(ulonglong2)), "alloc select");
        CK(dalloc(sc->allocs, q.rep, nn * sizeof(int)), "alloc select");
        CK(dalloc(sc->allocs, q.table, (size_t)ht * sizeof(int)), "alloc select");
        CK(dalloc(sc->allocs, q.rlist, nn * sizeof(int)), "alloc select");
        CK(dalloc(sc->allocs, q.rcount, 2 * sizeof(int)), "alloc select");
        CK(dalloc(sc->allocs, q.pcnt, nn * q.dmax * sizeof(int)), "alloc select");
        CK(dalloc(sc->allocs, q.ph, nn * sc->d.n_species * q.dmax * sc->es), "alloc select");
    }
    const size_t plane = (size_t)grid_c(sc).npad * sc->es;
    CK(dalloc(sc->allocs, sc->w_iso, q.dmax * plane), "alloc select weights");
    CK(dalloc(sc->allocs, sc->w_sun, q.dmax * plane), "alloc select weights");
    CK(cudaMemsetAsync(sc->w_iso, 0, q.dmax * plane, sc->st), "memset select weights");
    CK(cudaMemsetAsync(sc->w_sun, 0, q.dmax * plane, sc->st), "memset select weights");
    CK(cudaStreamSynchronize(sc->st), "sync");  // the host tables die here
    q.M = M;
    q.n_up = nup;
    q.rank = d_rank;
    q.lat = d_lat;
    q.latf = d_latf;
    q.glat = d_glat;
    q.glatf = d_glatf;
    q.dirf = d_dirf;
    q.grank = d_grank;
    q.gcell_start = d_gstart;
    q.gz = d_gz;
    q.gzsum = d_gzsum;
    q.gztot = gztot;
    sc->sel_ready = true;
    return TURSCA_OK;
}

// Row strides of the anisotropic mode's [nin][.] arrays: every row starts
// on 128 bytes (the tensor maps of the tensor-core kernel want 16).
inline int ani_ldx(const tk::GridC &g) { return (g.n_nodes + 31) / 32 * 32; }
inline int ani_ldz(const tk::GridC &g) { return (g.n_atm + 31) / 32 * 32; }

// Buffers of the anisotropic mode, allocated by its first assembly.
tursca_status ensure_aniso(tursca_scene *sc) {
    if (sc->ani_ready) return TURSCA_OK;
    const tk::GridC g = grid_c(sc);
    const size_t es = sc->es, nin = (size_t)g.nd + g.ngd, S = (size_t)g.S;
    const size_t nblk = (size_t)(g.nz + 1) * g.gpl;
    CK(dalloc(sc->allocs, sc->ani_Q, S * nin * g.nd * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_Qraw, S * nin * g.nd * sizeof(double)), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_SQ, (size_t)g.nz * S * nin * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_CT, (size_t)g.nd * g.n_atm * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_on, (size_t)g.n_atm * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_zf, nin * ani_ldz(g) * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_LsT, (size_t)g.nd * g.n_nodes * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_Wg, (size_t)std::max(1, g.n_ground) * std::max(1, g.ngd) * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_Lh, (size_t)g.nd * g.npad * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_CfH, (size_t)g.nd * g.npad * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_Pc, (size_t)sc->G.nval * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_b, nin * ani_ldx(g) * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_xtg, (size_t)std::max(1, g.n_ground) * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_xtb, (size_t)std::max(1, g.n_ground) * es), "alloc aniso");
    sc->ani_tables = false;
    CK(cudaMemsetAsync(sc->ani_CfH, 0, (size_t)g.nd * g.npad * es, sc->st), "memset aniso");
    CK(dalloc(sc->allocs, sc->ani_X, nin * ani_ldx(g) * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_Xn, nin * ani_ldx(g) * es), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_acc, 3 * sizeof(double)), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_part, 2 * nblk * sizeof(double)), "alloc aniso");
    CK(dalloc(sc->allocs, sc->ani_ctl, 4 * sizeof(int)), "alloc aniso");
    CK(cudaMemsetAsync(sc->ani_ctl, 0, 4 * sizeof(int), sc->st), "memset aniso");
    if (sc->d.precision != TURSCA_FP64) {
        // packed for the tile width the tensor-core launches use
        CK(dalloc(sc->allocs, sc->ani_Bl,
                  tk::ani_btab_floats((int)nin, tk::ani_leave_np(g.nd, g.S), g.S) * sizeof(float)),
           "alloc aniso");

    }
    CK(cudaMemsetAsync(sc->ani_Lh, 0, (size_t)g.nd * g.npad * es, sc->st), "memset aniso");
    sc->ani_ready = true;
    return TURSCA_OK;
}

// The FP32 refinement's buffers, allocated by the first refinement.
tursca_status ensure_aniso_refine(tursca_scene *sc) {
    if (sc->ani_X64) return TURSCA_OK;
    const tk::GridC g = grid_c(sc);
    const size_t nx = ((size_t)g.nd + g.ngd) * ani_ldx(g);
    CK(dalloc(sc->allocs, sc->ani_X64, nx * sizeof(float2)), "alloc aniso refinement");
    CK(dalloc(sc->allocs, sc->ani_L64, (size_t)g.nd * g.npad * sizeof(float2)), "alloc aniso refinement");
    CK(dalloc(sc->allocs, sc->ani_r, nx * sizeof(float)), "alloc aniso refinement");
    CK(dalloc(sc->allocs, sc->ani_E, nx * sizeof(float)), "alloc aniso refinement");
    {
        const int nin = g.nd + g.ngd, Kp = tk::ani_ds_kp(nin, g.S);
        const int jtop = std::max(0, g.nz - g.R) * g.nxy / tk::kAniTileM * tk::kAniTileM;
        CK(dalloc(sc->allocs, sc->ani_Ads, (size_t)Kp * ani_ldz(g) * sizeof(float2)), "alloc aniso refinement");
        CK(dalloc(sc->allocs, sc->ani_Atop, (size_t)Kp * tk::ani_ds_ldt(g, jtop) * sizeof(float2)),
           "alloc aniso refinement");
        CK(dalloc(sc->allocs, sc->ani_Bds, (size_t)Kp * 128 * sizeof(float)), "alloc aniso refinement");
    }
    CK(cudaMemsetAsync(sc->ani_L64, 0, (size_t)g.nd * g.npad * sizeof(float2), sc->st), "memset aniso");
    return TURSCA_OK;
}

template <typename T>
tk::AniP<T> ani_p(tursca_scene *sc) {
    tk::AniP<T> a;
    a.Q = (T *)sc->ani_Q;
    a.Qraw = sc->ani_Qraw;
    a.SQ = (T *)sc->ani_SQ;
    a.CT = (T *)sc->ani_CT;
    a.on = (T *)sc->ani_on;
    a.zf = (T *)sc->ani_zf;
    a.LsT = (T *)sc->ani_LsT;
    a.Wg = (T *)sc->ani_Wg;
    a.Lh = (T *)sc->ani_Lh;
    a.CfH = (T *)sc->ani_CfH;
    a.Pc = (T *)sc->ani_Pc;
    a.b = (T *)sc->ani_b;
    a.xtg = (T *)sc->ani_xtg;
    a.xtb = (T *)sc->ani_xtb;
    a.tslot = sc->ani_tslot;
    a.tseg = sc->ani_tseg;
    a.max_nt = sc->ani_max_nt;
    a.ldx = ani_ldx(grid_c(sc));
    a.ldz = ani_ldz(grid_c(sc));
    a.part = sc->ani_part;
    a.acc = sc->ani_acc;
    a.ctl = sc->ani_ctl;
    a.Bl = sc->ani_Bl;
    a.Ads = sc->ani_Ads;
    a.Atop = sc->ani_Atop;
    a.Bds = sc->ani_Bds;
    a.mma = sizeof(T) == 4 && sc->aniso == 1;
    return a;
}

// Terms of the series X <- radd + rho T L(X) (L with Lsun when `sun`) from
// the content of X (buffer 0) until the relative change is at most tol or
// max_terms terms: the stopping test runs on the device after every term and
// the host reads it every kAniCheck terms (the terms launched past the one
// that converged return at once).  Returns the buffer holding the
// last term in *xi (0: X, 1: Xn), the terms in *terms, the last change in *rel.
constexpr int kAniCheck = 16;
template <typename T>
tursca_status ani_series(tursca_scene *sc, T *X, T *Xn, const T *radd, bool sun, double tol, int max_terms,
                         int *xi, int *terms, double *rel, int term0 = 0) {
    const tk::GridC g = grid_c(sc);
    const tk::GraphP gp = graph_p(sc);
    const tk::FieldP<T> f = field_p<T>(sc);
    const tk::ViewC vc = view_c(sc);
    const tk::AniP<T> a = ani_p<T>(sc);
    T *buf[2] = {X, Xn};
    CK(cudaMemsetAsync(a.ctl, 0, 3 * sizeof(int), sc->st), "memset ctl");
    // terms term0 + 1, ...: term k reads buf[(k - 1 - term0) & 1]
    int k = 0, h[2] = {0, 0};
    double acc[3] = {0.0, 0.0, 1.0};
    max_terms -= term0;
    while (k < max_terms) {
        const int n = std::min(kAniCheck, max_terms - k);
        for (int i = 0; i < n; ++i, ++k) {
            const int p0 = prof_begin(sc, P_ALEAVE);
            CK(tk::launch_aniso_leave<T>(sc->st, g, gp, f, a, buf[k & 1], &sc->launches), "aniso term");
            prof_end(sc, p0);
            const int p1 = prof_begin(sc, P_AMOVE);
            tk::launch_aniso_move<T>(sc->st, g, gp, f, vc, a, buf[k & 1], buf[(k + 1) & 1], radd, sun, tol,
                                     term0 + k + 1, &sc->launches);
            prof_end(sc, p1);
        }
        CK(cudaGetLastError(), "aniso launch");
        CK(cudaMemcpyAsync(h, a.ctl, sizeof h, cudaMemcpyDeviceToHost, sc->st), "read ctl");
        CK(cudaMemcpyAsync(acc, a.acc, sizeof acc, cudaMemcpyDeviceToHost, sc->st), "read change");
        CK(cudaStreamSynchronize(sc->st), "sync");
        if (h[0]) break;
    }
    const int taken = h[0] ? h[1] - term0 : k;
    *xi = taken & 1;
    *terms = term0 + taken;
    *rel = acc[2];
    return TURSCA_OK;
}

// The series of Eq. fs_sum over the edge unknowns, then x and the emission
// from X.  FP64 scenes: until the relative change of X is at most rtol.
// FP32 scenes: the FP32 series to a change of max(rtol, 1e-6) (about the
// rounding floor of an FP32 iterate), then while the residual |F(X) - X| /
// |X|, evaluated in double-single (X in FP32 pairs), is above rtol, the
// correction series e = r + (F(e) - F(0)) and X += e in pairs.  (Chebyshev
// steps on a real interval, as the node form's refinements take, diverge
// here: the arrival-direction memory gives A a spectrum well off the real
// axis, and for a spectrum that fills a disk the plain series is the best
// polynomial method.)
constexpr int kAniMaxRefine = 8;
template <typename T>
tursca_status do_solve_aniso(tursca_scene *sc, int solver, double rtol, int max_iter, tursca_solve_info *info) {
    const tk::GridC g = grid_c(sc);
    const tk::FieldP<T> f = field_p<T>(sc);
    const int ldx = ani_ldx(g);
    const size_t nx = ((size_t)g.nd + g.ngd) * ldx;
    T *X = (T *)sc->ani_X, *Xn = (T *)sc->ani_Xn;
    // the first term from X = 0 is b, which the assembly formed (with the ground sums)
    CK(cudaMemcpyAsync(X, sc->ani_b, nx * sizeof(T), cudaMemcpyDeviceToDevice, sc->st), "copy b");
    CK(cudaMemcpyAsync(sc->ani_xtg, sc->ani_xtb, (size_t)std::max(1, g.n_ground) * sizeof(T),
                       cudaMemcpyDeviceToDevice, sc->st),
       "copy b");
    const double tol = sizeof(T) == 8 ? rtol : std::max(rtol, 1e-6);
    int xi = 0, terms = 0, total = 0, refinements = 0;
    double rel = 1.0;
    tursca_status e = ani_series<T>(sc, X, Xn, nullptr, true, tol, max_iter, &xi, &terms, &rel, 1);
    if (e) return e;
    total = terms;
    bool converged = rel <= tol;
    if constexpr (sizeof(T) == 4) {
        e = ensure_aniso_refine(sc);
        if (e) return e;
        const tk::GraphP gp = graph_p(sc);
        const tk::ViewC vc = view_c(sc);
        const tk::AniP<float> a = ani_p<float>(sc);
        tk::launch_aniso_update(sc->st, (long long)nx, xi ? Xn : X, sc->ani_X64, true);
        converged = false;
        while (refinements < kAniMaxRefine) {
            const int pr = prof_begin(sc, P_ARESID);
            tk::launch_aniso_resid(sc->st, g, gp, f, vc, a, sc->ani_X64, sc->ani_L64, sc->ani_r, &sc->launches);
            prof_end(sc, pr);
            sc->launches++;
            double acc[3];
            CK(cudaGetLastError(), "aniso residual launch");
            CK(cudaMemcpyAsync(acc, a.acc, sizeof acc, cudaMemcpyDeviceToHost, sc->st), "read residual");
            CK(cudaStreamSynchronize(sc->st), "sync");
            ++refinements;
            rel = acc[2];
            if (rel <= rtol) {
                converged = true;
                break;
            }
            if (total >= max_iter) break;
            // e = r + (F(e) - F(0)), from e = r
            const double tol_e = std::min(0.5, std::max(1e-6, 0.3 * rtol / rel));
            CK(cudaMemcpyAsync(sc->ani_E, sc->ani_r, nx * sizeof(float), cudaMemcpyDeviceToDevice, sc->st),
               "copy residual");
            int ei = 0, et = 0;
            double erel = 1.0;
            e = ani_series<float>(sc, sc->ani_E, (float *)Xn, sc->ani_r, false, tol_e, max_iter - total, &ei, &et,
                                  &erel);
            if (e) return e;
            total += et;
            tk::launch_aniso_update(sc->st, (long long)nx, ei ? (float *)Xn : sc->ani_E, sc->ani_X64, false);
        }
        tk::launch_aniso_finish<float, float2>(sc->st, g, f, sc->ani_X64, ldx, sc->x64, (float *)sc->emis,
                                               &sc->launches);
        sc->ani_Xsol = sc->ani_X64;
    } else {
        tk::launch_aniso_finish<T, T>(sc->st, g, f, xi ? Xn : X, ldx, sc->x64, (T *)sc->emis, &sc->launches);
        sc->ani_Xsol = xi ? Xn : X;
    }
    CK(cudaGetLastError(), "aniso launch");
    if (solver == TURSCA_SOLVER_AUTO)
        solver = sc->d.precision == TURSCA_FP64 ? TURSCA_SOLVER_GMRES : TURSCA_SOLVER_CHEBYSHEV;
    if (info) *info = tursca_solve_info{total, refinements, rel, 0.0, solver};
    e = sync_check(sc, "solve");
    if (e) return e;
    sc->solved = true;
    if (!converged) return fail(sc, TURSCA_E_NOT_CONVERGED, "series stopped above the tolerance");
    return TURSCA_OK;
}

extern "C" {

tursca_status tursca_scene_create(const tursca_grid_desc *desc, void *cuda_stream, tursca_scene **out) {
    if (!out) return fail(nullptr, TURSCA_E_INVALID, "out is null");
    *out = nullptr;
    std::string m = check_desc(desc);
    if (!m.empty()) return fail(nullptr, TURSCA_E_INVALID, m);
    tursca_scene *sc = new (std::nothrow) tursca_scene();
    if (!sc) return fail(nullptr, TURSCA_E_NOMEM, "host allocation failed");
    sc->d = *desc;
    sc->st = (cudaStream_t)cuda_stream;
    sc->es = desc->precision == TURSCA_FP64 ? 8 : 4;
    *out = sc;
    return TURSCA_OK;
}

tursca_status tursca_scene_destroy(tursca_scene *sc) {
    if (!sc) return TURSCA_OK;
    cudaStreamSynchronize(sc->st);
    free_list(sc->allocs);
    for (DevBuf &v : sc->vbuf)
        if (v.p) cudaFree(v.p);
    if (sc->hred) cudaFreeHost(sc->hred);
    if (sc->topk_hist_h) cudaFreeHost(sc->topk_hist_h);
    if (sc->bready) cudaEventDestroy(sc->bready);
    if (sc->bdone) cudaEventDestroy(sc->bdone);
    for (cudaEvent_t e : sc->ev) cudaEventDestroy(e);
    for (int i = 0; i < 3; ++i)
        if (sc->aux[i]) cudaStreamDestroy(sc->aux[i]);
    for (int i = 0; i < 5; ++i)
        if (sc->fork[i]) cudaEventDestroy(sc->fork[i]);
    delete sc;
    return TURSCA_OK;
}

tursca_status tursca_set_medium(tursca_scene *sc, const void *mu_abs, const void *mu_sca, const double *g,
                                double albedo) {
    const NvtxRange nvtx("tursca_set_medium");
    if (!sc) return fail(nullptr, TURSCA_E_INVALID, "scene is null");
    if (!mu_abs || !mu_sca || !g) return fail(sc, TURSCA_E_INVALID, "null field pointer");
    for (int s = 0; s < sc->d.n_species; ++s)
        if (!(std::fabs(g[s]) < 1.0)) return fail(sc, TURSCA_E_INVALID, "HG asymmetry must satisfy |g| < 1");
    if (!(albedo >= 0.0 && albedo <= 1.0)) return fail(sc, TURSCA_E_INVALID, "albedo must be in [0, 1]");
    tursca_status e = ensure_fields(sc);
    if (e) return e;
    const size_t na = (size_t)sc->d.nx * sc->d.ny * sc->d.nz;
    const int pm = prof_begin(sc, P_MEDIUM);
    CK(cudaMemcpyAsync(sc->mu_a, mu_abs, na * sc->es, cudaMemcpyDefault, sc->st), "copy mu_abs");
    CK(cudaMemcpyAsync(sc->mu_s, mu_sca, na * sc->es * sc->d.n_species, cudaMemcpyDefault, sc->st), "copy mu_sca");
    prof_end(sc, pm);
    CK(cudaMemsetAsync(sc->status, 0, sizeof(int), sc->st), "memset status");
    for (int s = 0; s < tk::MAX_SPECIES; ++s) sc->g[s] = s < sc->d.n_species ? g[s] : 0.0;
    sc->albedo = albedo;
    sc->medium = true;
    sc->assembled = sc->solved = sc->rendered = false;
    return TURSCA_OK;
}

tursca_status tursca_build_graph(tursca_scene *sc) {
    const NvtxRange nvtx("tursca_build_graph");
    if (!sc) return fail(nullptr, TURSCA_E_INVALID, "scene is null");
    if (sc->built) return TURSCA_OK;
    const tursca_grid_desc &d = sc->d;
    std::string m = tg::build_graph(sc->G, d.nx, d.ny, d.nz, d.hx, d.hy, d.hz, d.stencil_radius, d.fib_points);
    if (!m.empty()) return fail(sc, TURSCA_E_INVALID, m);
    tursca_status e = ensure_fields(sc);
    if (e) return e;
    tg::Graph &G = sc->G;
    // classes
    std::vector<tk::DClass> dc(G.classes.size());
    for (size_t i = 0; i < G.classes.size(); ++i) {
        const tg::SlotClass &c = G.classes[i];
        tk::DClass &o = dc[i];
        std::memset(&o, 0, sizeof(o));
        o.kind = (int16_t)c.kind;
        o.dir = (int16_t)std::max(c.dir, 0);
        o.hgdir = (int16_t)c.hgdir;
        o.k = (int16_t)c.k;
        o.bkind = (int16_t)c.bkind;
        o.up_idx = (int16_t)std::max(c.up_idx, 0);
        o.gdir = (int16_t)std::max(c.gdir, 0);
        o.c_one = (int16_t)c.c_one;
        o.pre_off = c.pre_off;
        o.seg_off = c.seg_off;
        o.hit_off = c.hit_off;
        o.pre_n = (int16_t)c.pre_n;
        o.seg_n = (int16_t)c.seg_n;
        o.hit_n = (int16_t)c.hit_n;
        o.n1_ground = (int16_t)c.n1_ground;
        o.n1_dx = (int16_t)c.n1_dx;
        o.n1_dy = (int16_t)c.n1_dy;
        o.n1_dz = (int16_t)c.n1_dz;
        o.dist1_inv = c.dist1 > 0 ? 1.0 / c.dist1 : 0.0;
        o.split = c.split;
        o.pre_tab = (int16_t)c.pre_tab;
        o.pre_dx = (int16_t)c.pre_dx;
        o.pre_dy = (int16_t)c.pre_dy;
        o.pre_dz = (int16_t)c.pre_dz;
        o.seg_tab = (int16_t)c.seg_tab;
        o.seg_dx = (int16_t)c.seg_dx;
        o.seg_dy = (int16_t)c.seg_dy;
        o.seg_dz = (int16_t)c.seg_dz;
        o.dist1_inv_f = (float)o.dist1_inv;
        o.split_f = (float)o.split;
    }
    CK(upload(sc, sc->allocs, sc->cls, dc.data(), dc.size() * sizeof(tk::DClass)), "upload classes");
    std::vector<tk::DTap> to;
    std::vector<float> lf;
    std::vector<double> ld;
    split_taps(G.taps, to, lf, ld);
    CK(upload(sc, sc->allocs, sc->taps, to.data(), to.size() * sizeof(tk::DTap)), "upload taps");
    CK(upload(sc, sc->allocs, sc->tlf, lf.data(), lf.size() * sizeof(float)), "upload taps");
    CK(upload(sc, sc->allocs, sc->tld, ld.data(), ld.size() * sizeof(double)), "upload taps");
    {
        std::vector<tk::RTap> rt;
        if (!ray_taps(G.taps, sc->d.nx, sc->d.ny, rt)) return fail(sc, TURSCA_E_INVALID, "grid too large for ray tables");
        CK(upload(sc, sc->allocs, sc->rtaps, rt.data(), std::max<size_t>(1, rt.size()) * sizeof(tk::RTap)), "upload taps");
        CK(cudaStreamSynchronize(sc->st), "sync");  // rt dies here
    }
    const int nd = (int)G.dirs.size(), ngd = (int)G.gdirs.size();
    std::vector<int4> dirs(nd);
    for (int u = 0; u < nd; ++u) dirs[u] = make_int4(G.dirs[u][0], G.dirs[u][1], G.dirs[u][2], G.kmax[u]);
    CK(upload(sc, sc->allocs, sc->dirs, dirs.data(), nd * sizeof(int4)), "upload dirs");
    CK(upload(sc, sc->allocs, sc->dir_len, G.len.data(), nd * sizeof(double)), "upload len");
    CK(upload(sc, sc->allocs, sc->q_iso, G.q_iso.data(), nd * sizeof(double)), "upload q");
    CK(upload(sc, sc->allocs, sc->q_lamb, G.q_lamb.data(), ngd * sizeof(double)), "upload q");
    std::vector<int4> gm(ngd);
    std::vector<double> gd1(ngd);
    for (int k = 0; k < ngd; ++k) {
        const auto &m0 = G.gdirs[k].mem[0];
        gm[k] = make_int4(m0[0], m0[1], m0[2], 0);
        double a = m0[0] * G.hx, b = m0[1] * G.hy, c = (m0[2] - 0.5) * G.hz;
        gd1[k] = std::sqrt(a * a + b * b + c * c);
    }
    CK(upload(sc, sc->allocs, sc->gmem1, gm.data(), ngd * sizeof(int4)), "upload gmem");
    CK(upload(sc, sc->allocs, sc->gdist1, gd1.data(), ngd * sizeof(double)), "upload gdist");
    {
        std::vector<float> a(G.len.begin(), G.len.end()), b(G.q_iso.begin(), G.q_iso.end()),
            c(G.q_lamb.begin(), G.q_lamb.end()), d(gd1.begin(), gd1.end());
        CK(upload(sc, sc->allocs, sc->dir_len_f, a.data(), a.size() * sizeof(float)), "upload f");
        CK(upload(sc, sc->allocs, sc->q_iso_f, b.data(), b.size() * sizeof(float)), "upload f");
        CK(upload(sc, sc->allocs, sc->q_lamb_f, c.data(), c.size() * sizeof(float)), "upload f");
        CK(upload(sc, sc->allocs, sc->gdist1_f, d.data(), d.size() * sizeof(float)), "upload f");
        CK(cudaStreamSynchronize(sc->st), "sync");  // the host vectors die here
    }
    CK(upload(sc, sc->allocs, sc->up_dirs, G.up_dirs.data(), G.up_dirs.size() * sizeof(int)), "upload up");
    CK(upload(sc, sc->allocs, sc->top_off, G.top_off.data(), G.top_off.size() * sizeof(int)), "upload top");
    CK(upload(sc, sc->allocs, sc->top_n, G.top_n.data(), G.top_n.size() * sizeof(int)), "upload top");
    CK(upload(sc, sc->allocs, sc->lat_off, G.lat_off.data(), nd * sizeof(int)), "upload lat");
    CK(upload(sc, sc->allocs, sc->lat_n, G.lat_n.data(), nd * sizeof(int)), "upload lat");
    CK(upload(sc, sc->allocs, sc->gtop_off, G.gtop_off.data(), ngd * sizeof(int)), "upload gtop");
    CK(upload(sc, sc->allocs, sc->gtop_n, G.gtop_n.data(), ngd * sizeof(int)), "upload gtop");
    std::vector<double> lat((size_t)3 * G.M);
    for (int i = 0; i < G.M; ++i)
        for (int a = 0; a < 3; ++a) lat[(size_t)3 * i + a] = G.lattice[G.cell_order[i]][a];
    CK(upload(sc, sc->allocs, sc->lattice, lat.data(), lat.size() * sizeof(double)), "upload lattice");
    CK(upload(sc, sc->allocs, sc->cell_start, G.cell_start.data(), G.cell_start.size() * sizeof(int)), "upload cells");
    std::vector<double> dh((size_t)3 * (nd + ngd));
    for (int u = 0; u < nd; ++u)
        for (int a = 0; a < 3; ++a) dh[3 * u + a] = G.uhat[u][a];
    for (int k = 0; k < ngd; ++k)
        for (int a = 0; a < 3; ++a) dh[3 * (nd + k) + a] = G.gdirs[k].uhat[a];
    CK(upload(sc, sc->allocs, sc->dirhat, dh.data(), dh.size() * sizeof(double)), "upload dirhat");
    // row templates (the CSR structure of K, one template per layer)
    std::vector<int4> tm(G.tmpl.size());
    for (size_t i = 0; i < G.tmpl.size(); ++i) {
        const tg::TSlot &t = G.tmpl[i];
        tm[i] = make_int4(t.cls, t.flat, (int)((unsigned)(t.sdx & 0xffff) | ((unsigned)(t.sdy & 0xffff) << 16)),
                          t.sz);
    }
    CK(upload(sc, sc->allocs, sc->tstart, G.tmpl_start.data(), G.tmpl_start.size() * sizeof(int)), "upload tmpl");
    CK(upload(sc, sc->allocs, sc->tmpl, tm.data(), tm.size() * sizeof(int4)), "upload tmpl");
    // the same templates as offsets in the solver's haloed layout (border R;
    // every template's column offset is at most R)
    {
        const int H = sc->d.stencil_radius, nxp = sc->d.nx + 2 * H, lp = nxp * (sc->d.ny + 2 * H);
        std::vector<int> tf(G.tmpl.size());
        for (int z = 0; z <= sc->d.nz; ++z)
            for (int i = G.tmpl_start[z]; i < G.tmpl_start[z + 1]; ++i) {
                const tg::TSlot &t = G.tmpl[i];
                if (std::abs(t.sdx) > H || std::abs(t.sdy) > H)
                    return fail(sc, TURSCA_E_INVALID, "internal error: template offset beyond the halo");
                const int szl = t.sz >= 0 ? t.sz : sc->d.nz;
                tf[i] = (szl - z) * lp + t.sdy * nxp + t.sdx;
            }
        CK(upload(sc, sc->allocs, sc->tflat, tf.data(), tf.size() * sizeof(int)), "upload tmpl");
        // gather tiles of the FP32 row-group passes (none when a group's
        // tile would exceed kTileMaxBytes)
        static_assert(tg::kTileLayers == tk::kTileLayers, "tile layers");
        tg::TileLayout tl;
        sc->tile_tl = 0;
        if (tg::tile_layout(G, H, tl).empty() &&
            (size_t)tk::kTileLayers * tl.tl * sizeof(float) <= (size_t)tk::kTileMaxBytes) {
            CK(upload(sc, sc->allocs, sc->ttile, tl.ttile.data(), tl.ttile.size() * sizeof(int)), "upload tiles");
            CK(upload(sc, sc->allocs, sc->tlay, tl.layers.data(), tl.layers.size() * sizeof(int)), "upload tiles");
            sc->tile_tl = tl.tl;
        }
        // edge-kernel descriptors (every lookup of a slot as one offset from
        // the receiver's haloed position)
        std::vector<tg::EdgeDesc> ed;
        std::vector<int> th, dh;
        const std::string err = tg::edge_descriptors(G, H, ed, th, dh);
        if (!err.empty()) return fail(sc, TURSCA_E_INVALID, "internal error: " + err);
        std::vector<tk::ASlot> as(ed.size());
        for (size_t i = 0; i < ed.size(); ++i) {
            const tg::EdgeDesc &e = ed[i];
            tk::ASlot &d = as[i];
            std::memset(&d, 0, sizeof(d));
            d.src = e.src;
            d.pre = e.pre;
            d.seg = e.seg;
            d.n1 = e.n1;
            d.aux = e.aux;
            d.tbase = e.tbase;
            // bit 12: the chain's first receiver is the receiver row itself;
            // bits 13-14: the edge kernel's straight-line kind of an
            // atmospheric source's chain node with table-read optical depths
            // (1: before the chain's end, 2: terminal with nothing beyond,
            // 3: terminal below the TOA), 0: the general code
            {
                const bool gs = (e.bits >> 11) & 1, cone = (e.bits >> 8) & 1, n1g = (e.bits >> 9) & 1;
                const bool n1_row = e.n1 == 0 && (gs || (!cone && !n1g));
                const int kind = e.bits & 15, bkind = (e.bits >> 4) & 15;
                const bool has_pre = (e.bits >> 10) & 1;
                int ft = 0;
                if (kind == 0 && !gs && !cone && !n1g && has_pre == !n1_row && (!has_pre || e.pre >= 0)) {
                    if (bkind == 0 && e.seg >= 0) ft = 1;
                    else if (bkind == 1) ft = 2;
                    else if (bkind == 2 && e.seg >= 0) ft = 3;
                }
                d.bits = e.bits | (n1_row ? 1 << 12 : 0) | (ft << 13);
            }
            d.dir = e.dir;
            d.hgdir = e.hgdir;
            d.taps = e.taps;
            d.pre_off = e.pre_off;
            d.seg_off = e.seg_off;
            d.hit_off = e.hit_off;
            d.q = (float)e.q;
            d.qd = e.q;
            d.dinv = (float)e.dinv;
            d.dinvd = e.dinv;
            d.split = (float)e.split;
            d.splitd = e.split;
        }
        CK(upload(sc, sc->allocs, sc->aslot, as.data(), as.size() * sizeof(tk::ASlot)), "upload slots");
        // the edge form's transport order: each layer's template slots
        // grouped by arrival direction (atmospheric direction, or nd + the
        // ground direction of a ground source), in template order inside a
        // direction
        {
            const int ndh = (int)G.uhat.size(), nin = ndh + (int)G.gdirs.size();
            std::vector<int4> perm(as.size());
            std::vector<int> segs((size_t)(sc->d.nz + 1) * (nin + 1));
            sc->ani_max_nt = 0;
            for (int z = 0; z <= sc->d.nz; ++z) {
                const int t0 = G.tmpl_start[z], nt = G.tmpl_start[z + 1] - t0;
                sc->ani_max_nt = std::max(sc->ani_max_nt, nt);
                std::vector<int> cnt(nin + 1, 0);
                for (int t = 0; t < nt; ++t) {
                    const tk::ASlot &d = as[t0 + t];
                    const int din = ((d.bits >> 11) & 1) ? ndh + d.dir : d.dir;
                    if (din < 0 || din >= nin) return fail(sc, TURSCA_E_INVALID, "internal error: arrival direction");
                    cnt[din + 1]++;
                }
                for (int w = 0; w < nin; ++w) cnt[w + 1] += cnt[w];
                for (int w = 0; w <= nin; ++w) segs[(size_t)z * (nin + 1) + w] = cnt[w];
                for (int t = 0; t < nt; ++t) {
                    const tk::ASlot &d = as[t0 + t];
                    const int din = ((d.bits >> 11) & 1) ? ndh + d.dir : d.dir;
                    perm[t0 + cnt[din]++] = make_int4(t, d.src, d.dir, 0);
                }
            }
            CK(upload(sc, sc->allocs, sc->ani_tslot, perm.data(), perm.size() * sizeof(int4)), "upload order");
            CK(upload(sc, sc->allocs, sc->ani_tseg, segs.data(), segs.size() * sizeof(int)), "upload order");
        }
        if (th.empty()) th.push_back(0);
        CK(upload(sc, sc->allocs, sc->tap_h, th.data(), th.size() * sizeof(int)), "upload taps");
        CK(upload(sc, sc->allocs, sc->dir_h, dh.data(), dh.size() * sizeof(int)), "upload dirs");
        CK(cudaStreamSynchronize(sc->st), "sync");
    }
    // Runs of the persistent streamed passes: one per SM, each an equal share
    // of the value stream cut at group boundaries (pass 0: all groups, pass
    // 1: the atmospheric layers)
    {
        int dev = 0, nsm = 0;
        CK(cudaGetDevice(&dev), "device");
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "device");
        const long long nxy = (long long)sc->d.nx * sc->d.ny;
        const int gpl = (int)((nxy + tk::kGroup - 1) / tk::kGroup);
        auto gstart = [&](long long gi) -> long long {
            const int z = (int)(gi / gpl), q = (int)(gi - (long long)z * gpl);
            if (z > sc->d.nz) return G.voff[sc->d.nz + 1];
            const long long nt = G.tmpl_start[z + 1] - G.tmpl_start[z];
            return G.voff[z] + (long long)q * nt * tk::kGroup;
        };
        for (int k = 0; k < 2; ++k) {
            const long long ng = (long long)(k == 0 ? sc->d.nz + 1 : sc->d.nz) * gpl;
            const int nb = (int)std::max<long long>(1, std::min<long long>(ng, std::max(nsm, 1)));
            const long long vtot = gstart(ng);
            std::vector<int> rg(nb + 1);
            std::vector<long long> rv(nb + 1);
            long long gi = 0;
            for (int b = 0; b <= nb; ++b) {
                const long long target = vtot * b / nb;
                while (gi < ng && gstart(gi) < target) ++gi;
                rg[b] = (int)gi;
                rv[b] = gstart(gi);
            }
            rg[nb] = (int)ng;
            rv[nb] = vtot;
            CK(upload(sc, sc->allocs, sc->run_g[k], rg.data(), rg.size() * sizeof(int)), "upload runs");
            CK(upload(sc, sc->allocs, sc->run_v[k], rv.data(), rv.size() * sizeof(long long)), "upload runs");
            sc->run_n[k] = nb;
        }
    }
    CK(upload(sc, sc->allocs, sc->voff, G.voff.data(), G.voff.size() * sizeof(long long)), "upload tmpl");
    CK(dalloc(sc->allocs, sc->val, (size_t)G.nval * sc->es), "alloc val");
    const size_t es = sc->es;
    CK(dalloc(sc->allocs, sc->tinf, (size_t)G.up_dirs.size() * G.n_atm * es), "alloc tinf");
    const size_t Hh = (size_t)sc->d.stencil_radius;
    const size_t lph = (sc->d.nx + 2 * Hh) * (sc->d.ny + 2 * Hh), nph = (size_t)(sc->d.nz + 1) * lph;
    CK(dalloc(sc->allocs, sc->tinfg, (size_t)ngd * lph * es), "alloc tinfg");
    CK(cudaMemsetAsync(sc->tinfg, 0, (size_t)ngd * lph * es, sc->st), "memset tinfg");
    CK(dalloc(sc->allocs, sc->q_sun, (size_t)sc->d.n_species * nd * es), "alloc qsun");
    sc->qt_ok = false;
    CK(dalloc(sc->allocs, sc->hgv, (size_t)sc->d.n_species * (nd + ngd) * es), "alloc hgv");
    CK(dalloc(sc->allocs, sc->hg0v, (size_t)sc->d.n_species * es), "alloc hg0v");
    CK(dalloc(sc->allocs, sc->cellsum, (size_t)sc->d.n_species * nd * sizeof(double)), "alloc cellsum");
    CK(upload(sc, sc->allocs, sc->canon_dirs, G.canon_dirs.data(), G.canon_dirs.size() * sizeof(int)), "upload canon");
    {
        // the taps of every canonical lattice segment, for the segment-table
        // kernel: each lies in the source's layer or the R above it and within
        // H columns and rows of it (the kernel's shared-memory tile)
        const int H = sc->d.stencil_radius;
        std::vector<int4> cs;
        std::vector<int> ct;
        for (int c = 0; c < (int)G.canon_dirs.size(); ++c) {
            const int u = G.canon_dirs[c];
            cs.push_back(make_int4((int)ct.size(), G.lat_n[u], G.dirs[u][2], 0));
            for (int k = 0; k < G.lat_n[u]; ++k) {
                const tg::Tap &t = G.taps[G.lat_off[u] + k];
                if (t.dz < 0 || t.dz > sc->d.stencil_radius || std::abs(t.dx) > H || std::abs(t.dy) > H)
                    return fail(sc, TURSCA_E_INVALID, "internal error: lattice tap outside the segment tile");
                ct.push_back(G.lat_off[u] + k);
            }
        }
        if (ct.size() > (size_t)tk::kSegMaxTaps || cs.size() > 64 || H > 2)
            return fail(sc, TURSCA_E_INVALID, "internal error: segment taps exceed the kernel's tables");
        if (G.dirs.size() > 128 || G.gdirs.size() > 128)
            return fail(sc, TURSCA_E_INVALID, "internal error: too many directions for the normaliser kernel");
        if (ct.empty()) ct.push_back(0);
        CK(upload(sc, sc->allocs, sc->cseg, cs.data(), cs.size() * sizeof(int4)), "upload canon");
        CK(upload(sc, sc->allocs, sc->ctap, ct.data(), ct.size() * sizeof(int)), "upload canon");
        sc->nctap = (int)(ct.size() == 1 && cs.empty() ? 0 : ct.size());
        // the same taps as kernel parameters, padded to tk::kSegTapsPer per
        // direction, at offsets into the kernel's tile (R + 1 layers of
        // (kSegTY + 2H) rows of kSegTX + 2H columns)
        const int TXh = tk::kSegTX + 2 * H, tpl = TXh * (tk::kSegTY + 2 * H);
        std::memset(&sc->segtab_f, 0, sizeof(sc->segtab_f));
        std::memset(&sc->segtab_d, 0, sizeof(sc->segtab_d));
        bool fits = cs.size() <= 64;
        for (size_t c = 0; c < cs.size() && fits; ++c) fits = cs[c].y <= tk::kSegTapsPer;
        if (fits) {
            for (size_t c = 0; c < cs.size(); ++c) {
                const int u = G.canon_dirs[c];
                sc->segtab_f.uz[c] = sc->segtab_d.uz[c] = G.dirs[u][2];
                for (int k = 0; k < cs[c].y; ++k) {
                    const tg::Tap &t = G.taps[G.lat_off[u] + k];
                    sc->segtab_f.off[c][k] = sc->segtab_d.off[c][k] = t.dz * tpl + t.dy * TXh + t.dx;
                    sc->segtab_f.len[c][k] = (float)t.len;
                    sc->segtab_d.len[c][k] = t.len;
                }
            }
            sc->segtab_f.n = sc->segtab_d.n = (int)cs.size();
        }
    }
    std::vector<int> upc(G.up_dirs.size());
    for (size_t i = 0; i < upc.size(); ++i) upc[i] = G.canon_of_dir[G.up_dirs[i]];
    CK(upload(sc, sc->allocs, sc->up_canon, upc.data(), upc.size() * sizeof(int)), "upload canon");
    CK(dalloc(sc->allocs, sc->tseg, G.canon_dirs.size() * nph * es), "alloc tseg");
    CK(cudaMemsetAsync(sc->tseg, 0, G.canon_dirs.size() * nph * es, sc->st), "memset tseg");
    CK(dalloc(sc->allocs, sc->rt, (size_t)G.n_atm * es), "alloc rt");
    CK(dalloc(sc->allocs, sc->wsp, (size_t)sc->d.n_species * G.n_atm * es), "alloc wsp");
    cudaError_t ce = cudaStreamSynchronize(sc->st);
    if (ce != cudaSuccess) return cuda_fail(sc, ce, "build_graph");
    if (sc->wq_auto) sc->wq = tk::choose_wq(grid_c(sc), sc->d.precision == TURSCA_FP64);
    for (int i = 0; i < 3; ++i) CK(cudaStreamCreateWithFlags(&sc->aux[i], cudaStreamNonBlocking), "aux stream");
    for (int i = 0; i < 5; ++i) CK(cudaEventCreateWithFlags(&sc->fork[i], cudaEventDisableTiming), "aux event");
    sc->built = true;
    return TURSCA_OK;
}

// The preselected maximum number of couplings K (Sec. 3): sc->c_eff becomes
// the (K + 1)-th largest FP64 coupling over every chain with a receiver (0
// when K reaches the count: the full stencil; the smallest positive double
// when that coupling is 0), found by a radix select over the chains' keys:
// six passes of at most 11 bits from the top, each a histogram over the keys
// that share the digits found so far, read back to pick the digit that
// holds the wanted rank.  Needs the fields of set_medium (the keys are
// formed from them before the rest of the assembly).
// The (K + 1)-th largest coupling, exactly as the FP64 couplings order (the
// oracle's arithmetic), in two steps.  A radix select on FP32 couplings
// (relative error of a few 1e-7) finds the FP32 value t of that rank; every
// coupling then differs from its FP32 value by far less than the band
// [t (1 - 1e-5), t (1 + 1e-5)], so the FP64 threshold lies in the band, the
// chains above it are all kept, and the threshold is the coupling of rank
// K + 1 - (chains above the band) among the band's chains, whose exact FP64
// keys are formed and ordered on the host.  Should that rank fall outside
// the band, the radix select runs on the FP64 keys of every chain instead.
tursca_status topk_threshold(tursca_scene *sc, const tk::GridC &g, const tk::GraphP &gp) {
    const long long tot = (long long)g.n_atm * g.nd + (long long)g.n_ground * g.ngd;
    if (!sc->topk_keys) {
        CK(dalloc(sc->allocs, sc->topk_keys, (size_t)tot * sizeof(unsigned long long)), "alloc topk keys");
        CK(dalloc(sc->allocs, sc->topk_hist, sizeof(unsigned int) << tk::kTopkDigitBits), "alloc topk hist");
        CK(dalloc(sc->allocs, sc->topk_band, (size_t)tot * sizeof(int)), "alloc topk band");
        CK(dalloc(sc->allocs, sc->topk_cnt, 2 * sizeof(int)), "alloc topk band");
        cudaError_t e = cudaMallocHost((void **)&sc->topk_hist_h, sizeof(unsigned int) << tk::kTopkDigitBits);
        if (e != cudaSuccess) return cuda_fail(sc, e, "alloc pinned");
    }
    if (!sc->selp.musmax_bits) {
        tursca_status e = ensure_select(sc);
        if (e) return e;
    }
    const bool fp64 = sc->d.precision == TURSCA_FP64;
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev), "device");
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "device");
    const int nb = std::max(1, nsm) * 8;
    const int nbins = 1 << tk::kTopkDigitBits;
    const long long want = sc->max_couplings + 1;  // wanted rank from the top (1-based)
    auto set_threshold = [&](unsigned long long key) {
        double thr;
        const unsigned long long bits = key - 1ull;
        std::memcpy(&thr, &bits, sizeof(thr));
        sc->c_eff = thr > 0.0 ? thr : 4.9406564584124654e-324;  // a zero coupling: keep C > 0
    };
    // one radix pass: the histogram of the next digit, read back
    auto hist_pass = [&](auto launch) -> tursca_status {
        launch();
        sc->launches += 1;
        CK(cudaMemcpyAsync(sc->topk_hist_h, sc->topk_hist, sizeof(unsigned int) * nbins, cudaMemcpyDeviceToHost,
                           sc->st), "d2h");
        CK(cudaStreamSynchronize(sc->st), "sync");
        return TURSCA_OK;
    };
    // ---- FP32 couplings: radix select over 32-bit keys
    unsigned int *keys32 = reinterpret_cast<unsigned int *>(sc->topk_keys);
    if (fp64)
        tk::launch_topk_keys32<double>(sc->st, g, gp, field_p<double>(sc), view_c(sc), sc->selp.musmax_bits, keys32,
                                       &sc->launches);
    else
        tk::launch_topk_keys32<float>(sc->st, g, gp, field_p<float>(sc), view_c(sc), sc->selp.musmax_bits, keys32,
                                      &sc->launches);
    unsigned int prefix32 = 0u;
    long long rank = want;
    for (int hi = 32, pass = 0; hi > 0; ++pass) {
        const int width = std::min(tk::kTopkDigitBits, hi), shift = hi - width;
        tursca_status e = hist_pass([&] {
            tk::launch_topk_hist32(sc->st, keys32, tot, shift, width, hi, prefix32, sc->topk_hist, nb);
        });
        if (e) return e;
        const unsigned int *h = sc->topk_hist_h;
        if (pass == 0) {
            long long count = 0;
            for (int b = 0; b < nbins; ++b) count += h[b];
            sc->n_couplings = count;
            if (sc->max_couplings >= count) {
                sc->c_eff = 0.0;
                sc->n_kept = count;
                return TURSCA_OK;
            }
        }
        long long acc = 0;
        int pick = -1;
        for (int b = (1 << width) - 1; b >= 0; --b) {
            if (acc + (long long)h[b] >= rank) {
                pick = b;
                break;
            }
            acc += h[b];
        }
        if (pick < 0) return fail(sc, TURSCA_E_INVALID, "internal error: coupling rank not found");
        rank -= acc;
        prefix32 = (prefix32 << width) | (unsigned int)pick;
        hi = shift;
    }
    float t32;
    {
        const unsigned int bits = prefix32 - 1u;
        std::memcpy(&t32, &bits, sizeof(t32));
    }
    // ---- the band around it: exact keys of its chains, ordered on the host
    const double lo = (double)t32 * (1.0 - 1e-5), hi = (double)t32 * (1.0 + 1e-5);
    tk::launch_topk_band(sc->st, keys32, tot, lo, hi, sc->topk_band, sc->topk_cnt, nb);
    int cnt[2] = {0, 0};
    CK(cudaMemcpyAsync(cnt, sc->topk_cnt, sizeof cnt, cudaMemcpyDeviceToHost, sc->st), "d2h");
    CK(cudaStreamSynchronize(sc->st), "sync");
    const long long nband = cnt[0], above = cnt[1], rb = want - above;
    if (rb >= 1 && rb <= nband) {
        if (fp64)
            tk::launch_topk_band_keys<double>(sc->st, g, gp, field_p<double>(sc), view_c(sc), sc->selp.musmax_bits,
                                              sc->topk_band, (int)nband, sc->topk_keys);
        else
            tk::launch_topk_band_keys<float>(sc->st, g, gp, field_p<float>(sc), view_c(sc), sc->selp.musmax_bits,
                                             sc->topk_band, (int)nband, sc->topk_keys);
        sc->launches += 2;
        std::vector<unsigned long long> v((size_t)nband);
        CK(cudaMemcpyAsync(v.data(), sc->topk_keys, (size_t)nband * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, sc->st), "d2h");
        CK(cudaStreamSynchronize(sc->st), "sync");
        std::nth_element(v.begin(), v.begin() + (rb - 1), v.end(), std::greater<unsigned long long>());
        const unsigned long long key = v[(size_t)rb - 1];
        long long above_key = 0;
        for (unsigned long long k : v) above_key += k > key;
        sc->n_kept = above + above_key;
        set_threshold(key);
        return TURSCA_OK;
    }
    // ---- otherwise: the radix select over the FP64 keys of every chain
    if (fp64)
        tk::launch_topk_keys<double>(sc->st, g, gp, field_p<double>(sc), view_c(sc), sc->selp.musmax_bits,
                                     sc->topk_keys, &sc->launches);
    else
        tk::launch_topk_keys<float>(sc->st, g, gp, field_p<float>(sc), view_c(sc), sc->selp.musmax_bits,
                                    sc->topk_keys, &sc->launches);
    unsigned long long prefix = 0ull;
    rank = want;
    sc->n_kept = 0;
    for (int hi64 = 64; hi64 > 0;) {
        const int width = std::min(tk::kTopkDigitBits, hi64), shift = hi64 - width;
        tursca_status e = hist_pass([&] {
            tk::launch_topk_hist(sc->st, sc->topk_keys, tot, shift, width, hi64, prefix, sc->topk_hist, nb);
        });
        if (e) return e;
        const unsigned int *h = sc->topk_hist_h;
        long long acc = 0;
        int pick = -1;
        for (int b = (1 << width) - 1; b >= 0; --b) {
            if (acc + (long long)h[b] >= rank) {
                pick = b;
                break;
            }
            acc += h[b];
        }
        if (pick < 0) return fail(sc, TURSCA_E_INVALID, "internal error: coupling rank not found");
        rank -= acc;
        sc->n_kept += acc;  // keys in higher bins: couplings above the threshold
        prefix = (prefix << width) | (unsigned long long)pick;
        hi64 = shift;
    }
    set_threshold(prefix);
    return TURSCA_OK;
}

tursca_status tursca_assemble_flux(tursca_scene *sc, const tursca_geometry *geom) {
    const NvtxRange nvtx("tursca_assemble_flux");
    if (!sc) return fail(nullptr, TURSCA_E_INVALID, "scene is null");
    if (!geom) return fail(sc, TURSCA_E_INVALID, "geometry is null");
    if (!sc->built) return fail(sc, TURSCA_E_STATE, "build_graph has not been called");
    if (!sc->medium) return fail(sc, TURSCA_E_STATE, "set_medium has not been called");
    if (!(geom->f0 > 0.0) || !std::isfinite(geom->f0)) return fail(sc, TURSCA_E_INVALID, "f0 must be positive");
    if (sc->aniso && (sc->single || sc->c_min > 0.0 || sc->max_couplings > 0))
        return fail(sc, TURSCA_E_INVALID,
                    "the anisotropic mode combines with neither single scattering nor coupling selection");
    if (sc->c_min > 0.0 && sc->max_couplings > 0)
        return fail(sc, TURSCA_E_INVALID, "c_min and a maximum number of couplings exclude each other");
    bool same = sc->view_ok && geom->sza == sc->geom.sza && geom->saa == sc->geom.saa && geom->vza == sc->geom.vza &&
                geom->vaa == sc->geom.vaa && geom->npx == sc->geom.npx && geom->npy == sc->geom.npy;
    if (!same) {
        tg::ViewTables VT;
        std::string m = tg::build_view(sc->G, VT, geom->sza, geom->saa, geom->vza, geom->vaa, geom->npx, geom->npy);
        if (!m.empty()) return fail(sc, TURSCA_E_INVALID, m);
        for (const auto &t : VT.sun_taps)
            if (std::abs(t.dx) > 32000 || std::abs(t.dy) > 32000) return fail(sc, TURSCA_E_INVALID, "ray too oblique");
        for (const auto &t : VT.los_taps)
            if (std::abs(t.dx) > 32000 || std::abs(t.dy) > 32000) return fail(sc, TURSCA_E_INVALID, "ray too oblique");
        CK(cudaStreamSynchronize(sc->st), "sync");  // earlier work of the scene may read the buffers
        sc->VT = VT;
        std::vector<tk::DTap> to;
        std::vector<float> lf;
        std::vector<double> ld;
        DevBuf *vb = sc->vbuf;
        split_taps(VT.sun_taps, to, lf, ld);
        CK(put(vb[VB_SUN_TAPS], sc->sun_taps, to.data(), to.size() * sizeof(tk::DTap), sc->st), "upload sun");
        CK(put(vb[VB_SUN_LF], sc->sun_lf, lf.data(), lf.size() * sizeof(float), sc->st), "upload sun");
        CK(put(vb[VB_SUN_LD], sc->sun_ld, ld.data(), ld.size() * sizeof(double), sc->st), "upload sun");
        CK(put(vb[VB_SUN_OFF], sc->sun_off, VT.sun_off.data(), VT.sun_off.size() * sizeof(int), sc->st), "upload sun");
        CK(put(vb[VB_SUN_N], sc->sun_n, VT.sun_n.data(), VT.sun_n.size() * sizeof(int), sc->st), "upload sun");
        {
            std::vector<tk::RTap> rt;
            if (!ray_taps(VT.sun_taps, sc->d.nx, sc->d.ny, rt)) return fail(sc, TURSCA_E_INVALID, "grid too large for ray tables");
            CK(put(vb[VB_SUN_RT], sc->sun_rt, rt.data(), std::max<size_t>(1, rt.size()) * sizeof(tk::RTap), sc->st), "upload sun");
            CK(cudaStreamSynchronize(sc->st), "sync");  // rt dies here
        }
        // (pageable host memory: the copies are complete when put returns)
        split_taps(VT.los_taps, to, lf, ld);
        CK(put(vb[VB_LOS_TAPS], sc->los_taps, to.data(), to.size() * sizeof(tk::DTap), sc->st), "upload los");
        CK(put(vb[VB_LOS_LF], sc->los_lf, lf.data(), lf.size() * sizeof(float), sc->st), "upload los");
        CK(put(vb[VB_LOS_LD], sc->los_ld, ld.data(), ld.size() * sizeof(double), sc->st), "upload los");
        CK(put(vb[VB_LOS_OFF], sc->los_off, VT.los_off.data(), VT.los_off.size() * sizeof(int), sc->st), "upload los");
        CK(put(vb[VB_LOS_N], sc->los_n, VT.los_n.data(), VT.los_n.size() * sizeof(int), sc->st), "upload los");
        CK(put(vb[VB_PIX_CX], sc->pix_cx, VT.pix_cx.data(), VT.pix_cx.size() * sizeof(int), sc->st), "upload pix");
        CK(put(vb[VB_PIX_CY], sc->pix_cy, VT.pix_cy.data(), VT.pix_cy.size() * sizeof(int), sc->st), "upload pix");
        CK(put(vb[VB_PIX_CLS], sc->pix_cls, VT.pix_cls.data(), VT.pix_cls.size() * sizeof(int), sc->st), "upload pix");
        size_t np = (size_t)geom->npx * geom->npy;
        CK(put(vb[VB_RAD], sc->rad, nullptr, np * sc->es, sc->st), "alloc rad");
        CK(put(vb[VB_REFL], sc->refl, nullptr, np * sc->es, sc->st), "alloc refl");
        CK(cudaStreamSynchronize(sc->st), "sync");
        sc->view_ok = true;
    }
    sc->geom = *geom;
    const tk::GridC g = grid_c(sc);
    const tk::GraphP gp = graph_p(sc);
    const tk::ViewC vc = view_c(sc);
    const tk::ViewP vp = view_p(sc);
    if (sc->single) {
        // first scattering order: the direct beam and the phase tables only
        int pd = prof_begin(sc, P_PRE);
        if (sc->d.precision == TURSCA_FP64)
            tk::launch_assemble_direct<double>(sc->st, g, field_p<double>(sc), vc, vp, &sc->launches);
        else
            tk::launch_assemble_direct<float>(sc->st, g, field_p<float>(sc), vc, vp, &sc->launches);
        prof_end(sc, pd);
        CK(cudaMemsetAsync(sc->s, 0, (size_t)sc->G.n_nodes * sc->es, sc->st), "memset s");
        CK(cudaMemsetAsync(sc->gsun, 0, (size_t)sc->G.n_atm * sc->es, sc->st), "memset gsun");
        CK(cudaGetLastError(), "assemble launch");
        sc->single_asm = sc->assembled = true;
        sc->sel_asm = sc->aniso_asm = false;
        sc->solved = sc->rendered = false;
        return TURSCA_OK;
    }
    int p0 = prof_begin(sc, P_PRE);
    const cudaStream_t streams[4] = {sc->st, sc->aux[0], sc->aux[1], sc->aux[2]};
    double key[6 + tk::MAX_SPECIES] = {vc.s0[0], vc.s0[1], vc.s0[2], vc.v[0], vc.v[1], vc.v[2]};
    for (int sp = 0; sp < tk::MAX_SPECIES; ++sp) key[6 + sp] = sp < g.S ? vc.g[sp] : 0.0;
    bool tables = !sc->qt_ok;
    for (int k = 0; k < 6 + tk::MAX_SPECIES; ++k) tables = tables || key[k] != sc->qt_key[k];
    if (sc->d.precision == TURSCA_FP64)
        tk::launch_assemble_pre<double>(streams, sc->fork, g, gp, field_p<double>(sc), vc, vp, sc->segtab_d, tables,
                                        &sc->launches);
    else
        tk::launch_assemble_pre<float>(streams, sc->fork, g, gp, field_p<float>(sc), vc, vp, sc->segtab_f, tables,
                                       &sc->launches);
    sc->qt_ok = true;
    for (int k = 0; k < 6 + tk::MAX_SPECIES; ++k) sc->qt_key[k] = key[k];
    prof_end(sc, p0);
    sc->c_eff = sc->c_min;
    sc->n_couplings = sc->n_kept = -1;
    if (sc->max_couplings > 0) {
        tursca_status e = topk_threshold(sc, g, gp);
        if (e) return e;
    }
    if (sc->c_eff > 0.0) {
        tursca_status e = ensure_select(sc);
        if (e) return e;
        tk::SelP q = sc->selp;
        q.c_min = sc->c_eff;
        int ps = prof_begin(sc, P_SEL);
        if (sc->d.precision == TURSCA_FP64)
            tk::launch_select<double>(sc->st, g, gp, field_p<double>(sc), vc, vp, q, (double *)sc->w_iso,
                                      (double *)sc->w_sun, &sc->launches);
        else
            tk::launch_select<float>(sc->st, g, gp, field_p<float>(sc), vc, vp, q, (float *)sc->w_iso,
                                     (float *)sc->w_sun, &sc->launches);
        prof_end(sc, ps);
        int p1 = prof_begin(sc, P_ROWS);
        if (sc->d.precision == TURSCA_FP64)
            tk::launch_assemble_rows_sel<double>(sc->st, g, gp, field_p<double>(sc), vc, (const double *)sc->w_iso,
                                                 (const double *)sc->w_sun, &sc->launches);
        else
            tk::launch_assemble_rows_sel<float>(sc->st, g, gp, field_p<float>(sc), vc, (const float *)sc->w_iso,
                                                (const float *)sc->w_sun, &sc->launches);
        prof_end(sc, p1);
    } else if (sc->aniso) {
        tursca_status e = ensure_aniso(sc);
        if (e) return e;
        int p1 = prof_begin(sc, P_ROWS);
        // the quadrature tables depend on the HG asymmetries (and the graph) only
        bool tables = !sc->ani_tables;
        for (int sp = 0; sp < g.S; ++sp) tables = tables || vc.g[sp] != sc->ani_g[sp];
        if (sc->d.precision == TURSCA_FP64) {
            tk::launch_assemble_rows_p<double>(sc->st, g, gp, field_p<double>(sc), vc, &sc->launches);
            tk::launch_aniso_prep<double>(sc->st, g, gp, field_p<double>(sc), vc, vp, ani_p<double>(sc), tables,
                                          &sc->launches);
        } else {
            tk::launch_assemble_rows_p<float>(sc->st, g, gp, field_p<float>(sc), vc, &sc->launches);
            tk::launch_aniso_prep<float>(sc->st, g, gp, field_p<float>(sc), vc, vp, ani_p<float>(sc), tables,
                                         &sc->launches);
        }
        sc->ani_tables = true;
        for (int sp = 0; sp < g.S; ++sp) sc->ani_g[sp] = vc.g[sp];
        prof_end(sc, p1);
    } else {
        int p1 = prof_begin(sc, P_ROWS);
        if (sc->d.precision == TURSCA_FP64)
            tk::launch_assemble_rows<double>(sc->st, g, gp, field_p<double>(sc), vc, &sc->launches);
        else
            tk::launch_assemble_rows<float>(sc->st, g, gp, field_p<float>(sc), vc, &sc->launches);
        prof_end(sc, p1);
    }
    sc->sel_asm = sc->c_eff > 0.0;
    sc->aniso_asm = sc->aniso != 0;
    CK(cudaGetLastError(), "assemble launch");
    sc->assembled = true;
    sc->single_asm = false;
    sc->solved = sc->rendered = false;
    return TURSCA_OK;
}

tursca_status tursca_solve_with(tursca_scene *sc, int solver, double rtol, int max_iter, tursca_solve_info *info) {
    const NvtxRange nvtx("tursca_solve");
    if (!sc) return fail(nullptr, TURSCA_E_INVALID, "scene is null");
    if (!sc->assembled) return fail(sc, TURSCA_E_STATE, "assemble_flux has not been called");
    if (!(rtol > 0.0) || max_iter < 1) return fail(sc, TURSCA_E_INVALID, "rtol must be > 0 and max_iter >= 1");
    sc->rendered = false;
    if (solver < 0 || solver > 3) return fail(sc, TURSCA_E_INVALID, "unknown solver");
    // The node-form solve queues its first passes behind the assembly without
    // waiting for it: the status word that reports invalid fields comes back
    // with the solve's first residual norm.  The other forms check it now.
    if (sc->single_asm || sc->aniso_asm) {
        tursca_status e = sync_check(sc, "assemble");
        if (e) return e;
    } else {
        CK(cudaGetLastError(), "assemble");
    }
    if (sc->single_asm) {
        // s = 0: x = 0 solves the system exactly, with no products with K
        const size_t H = (size_t)sc->d.stencil_radius;
        const size_t np = (size_t)(sc->d.nz + 1) * (sc->d.nx + 2 * H) * (sc->d.ny + 2 * H);
        CK(cudaMemsetAsync(sc->x64, 0, np * sizeof(double), sc->st), "memset x");
        if (solver == TURSCA_SOLVER_AUTO)
            solver = sc->d.precision == TURSCA_FP64 ? TURSCA_SOLVER_GMRES : TURSCA_SOLVER_CHEBYSHEV;
        if (info) *info = tursca_solve_info{0, 0, 0.0, 0.0, solver};
        sc->solved = true;
        return TURSCA_OK;
    }
    const int ps = prof_begin(sc, P_SOLVE);
    tursca_status r;
    if (sc->aniso_asm)
        r = sc->d.precision == TURSCA_FP64 ? do_solve_aniso<double>(sc, solver, rtol, max_iter, info)
                                           : do_solve_aniso<float>(sc, solver, rtol, max_iter, info);
    else
        r = sc->d.precision == TURSCA_FP64
                ? do_solve<double>(sc, solver, rtol, max_iter, info, forward_io<double>(sc))
                : do_solve<float>(sc, solver, rtol, max_iter, info, forward_io<float>(sc));
    prof_end(sc, ps);
    return r;
}

tursca_status tursca_solve(tursca_scene *sc, double rtol, int max_iter, tursca_solve_info *info) {
    return tursca_solve_with(sc, TURSCA_SOLVER_AUTO, rtol, max_iter, info);
}

tursca_status tursca_render_radiance(tursca_scene *sc, void *radiance, void *reflectance) {
    const NvtxRange nvtx("tursca_render_radiance");
    if (!sc) return fail(nullptr, TURSCA_E_INVALID, "scene is null");
    if (!sc->solved) return fail(sc, TURSCA_E_STATE, "solve has not been called");
    if (sc->d.precision == TURSCA_FP64) return do_render<double>(sc, radiance, reflectance);
    return do_render<float>(sc, radiance, reflectance);
}

tursca_status tursca_run(tursca_scene *sc, const void *mu_abs, const void *mu_sca, const double *g, double albedo,
                         const tursca_geometry *geom, int solver, double rtol, int max_iter, void *radiance,
                         void *reflectance, tursca_solve_info *info) {
    const NvtxRange nvtx("tursca_run");
    tursca_status e = tursca_set_medium(sc, mu_abs, mu_sca, g, albedo);
    if (e) return e;
    e = tursca_assemble_flux(sc, geom);
    if (e) return e;
    e = tursca_solve_with(sc, solver, rtol, max_iter, info);
    if (e) return e;
    return tursca_render_radiance(sc, radiance, reflectance);
}

tursca_status tursca_adjoint(tursca_scene *sc, const void *dJ_dL, void *dJ_dmu_abs) {
    const NvtxRange nvtx("tursca_adjoint");
    if (!sc) return fail(nullptr, TURSCA_E_INVALID, "scene is null");
    if (!dJ_dL || !dJ_dmu_abs) return fail(sc, TURSCA_E_INVALID, "dJ_dL and dJ_dmu_abs must not be null");
    if (!sc->rendered) return fail(sc, TURSCA_E_STATE, "render_radiance has not been called since the last solve");
    if (sc->single_asm) return fail(sc, TURSCA_E_STATE, "the adjoint needs a multiple-scattering assembly");
    if (sc->aniso_asm) return fail(sc, TURSCA_E_UNSUPPORTED, "the adjoint does not cover the anisotropic mode");
    tursca_status e = ensure_adjoint(sc);
    if (e) return e;
    if (sc->d.precision == TURSCA_FP64) return do_adjoint<double>(sc, dJ_dL, dJ_dmu_abs);
    return do_adjoint<float>(sc, dJ_dL, dJ_dmu_abs);
}

tursca_status tursca_get(tursca_scene *sc, tursca_field which, void *dst, size_t bytes) {
    if (!sc) return fail(nullptr, TURSCA_E_INVALID, "scene is null");
    if (!dst) return fail(sc, TURSCA_E_INVALID, "dst is null");
    if (!sc->built) return fail(sc, TURSCA_E_STATE, "build_graph has not been called");
    const tg::Graph &G = sc->G;
    const size_t es = sc->es, nn = (size_t)G.n_nodes, na = (size_t)G.n_atm, nnz = (size_t)G.nnz;
    const void *src = nullptr;
    size_t need = 0;
    bool host = false;
    std::vector<int32_t> tmp32;
    void *dtmp = nullptr;
    switch (which) {
        case TURSCA_F_ROW_PTR:
        case TURSCA_F_COL:
        case TURSCA_F_VAL:
        case TURSCA_F_SLOT_DIR:
        case TURSCA_F_SLOT_K: {
            // CSR view of the slot-major matrix, produced on demand
            need = which == TURSCA_F_ROW_PTR ? (nn + 1) * 4
                   : which == TURSCA_F_COL   ? nnz * 4
                   : which == TURSCA_F_VAL   ? nnz * es
                   : which == TURSCA_F_SLOT_DIR ? nnz * 2
                                                : nnz;
            if (bytes != need) return fail(sc, TURSCA_E_INVALID, "bytes does not match the field size");
            if (which == TURSCA_F_VAL && (!sc->assembled || sc->single_asm || sc->aniso_asm))
                return fail(sc, TURSCA_E_STATE, "K is not assembled");
            CK(cudaMalloc(&dtmp, need), "alloc");
            const tk::GridC gc = grid_c(sc);
            const tk::GraphP gp = graph_p(sc);
            int32_t *rp = which == TURSCA_F_ROW_PTR ? (int32_t *)dtmp : nullptr;
            int32_t *cc = which == TURSCA_F_COL ? (int32_t *)dtmp : nullptr;
            int16_t *dd = which == TURSCA_F_SLOT_DIR ? (int16_t *)dtmp : nullptr;
            int8_t *kk = which == TURSCA_F_SLOT_K ? (int8_t *)dtmp : nullptr;
            if (sc->d.precision == TURSCA_FP64)
                tk::launch_export_csr<double>(sc->st, gc, gp, (const double *)sc->val, rp, cc,
                                              which == TURSCA_F_VAL ? (double *)dtmp : nullptr, dd, kk);
            else
                tk::launch_export_csr<float>(sc->st, gc, gp, (const float *)sc->val, rp, cc,
                                             which == TURSCA_F_VAL ? (float *)dtmp : nullptr, dd, kk);
            sc->launches++;
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst, dtmp, need, cudaMemcpyDefault, sc->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(sc->st);
            cudaFree(dtmp);
            if (e != cudaSuccess) return cuda_fail(sc, e, "get csr");
            return TURSCA_OK;
        }
        case TURSCA_F_TSUN: src = sc->tsun; need = nn * es; break;
        case TURSCA_F_E1: src = sc->e1; need = nn * es; break;
        case TURSCA_F_S: src = sc->s; need = nn * es; break;
        case TURSCA_F_X:
            // the solver keeps x haloed: gather the nodes into the residual
            // buffer (scratch between solves) first
            if (!sc->fields_alloc) return fail(sc, TURSCA_E_STATE, "set_medium has not been called");
            tk::launch_from_halo<double>(sc->st, grid_c(sc), sc->x64, sc->r64);
            src = sc->r64;
            need = nn * 8;
            break;
        case TURSCA_F_EMIS: src = sc->emis; need = na * es; break;
        case TURSCA_F_GSUN: src = sc->gsun; need = na * es; break;
        case TURSCA_F_Q_ISO: src = G.q_iso.data(); need = G.q_iso.size() * 8; host = true; break;
        case TURSCA_F_Q_LAMB: src = G.q_lamb.data(); need = G.q_lamb.size() * 8; host = true; break;
        case TURSCA_F_Q_SUN: src = sc->q_sun; need = (size_t)sc->d.n_species * G.dirs.size() * es; break;
        case TURSCA_F_ANISO_X: {
            // the edge unknowns of the last anisotropic solve, [nin][n_nodes] FP64
            if (!sc->solved || !sc->aniso_asm || !sc->ani_Xsol)
                return fail(sc, TURSCA_E_STATE, "no anisotropic solve");
            const tk::GridC gc = grid_c(sc);
            const size_t nx = ((size_t)gc.nd + gc.ngd) * gc.n_nodes;
            if (bytes != nx * 8) return fail(sc, TURSCA_E_INVALID, "bytes does not match the field size");
            void *dtmp = nullptr;
            CK(cudaMalloc(&dtmp, nx * 8), "alloc");
            if (sc->d.precision == TURSCA_FP64)
                tk::launch_aniso_export<double>(sc->st, gc, (const double *)sc->ani_Xsol, ani_ldx(gc), (double *)dtmp);
            else
                tk::launch_aniso_export<float2>(sc->st, gc, (const float2 *)sc->ani_Xsol, ani_ldx(gc), (double *)dtmp);
            sc->launches++;
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst, dtmp, nx * 8, cudaMemcpyDefault, sc->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(sc->st);
            cudaFree(dtmp);
            if (e != cudaSuccess) return cuda_fail(sc, e, "get aniso X");
            return TURSCA_OK;
        }
        case TURSCA_F_DIRS:
            tmp32.resize(G.dirs.size() * 3);
            for (size_t u = 0; u < G.dirs.size(); ++u)
                for (int a = 0; a < 3; ++a) tmp32[3 * u + a] = G.dirs[u][a];
            src = tmp32.data();
            need = tmp32.size() * 4;
            host = true;
            break;
        default: return fail(sc, TURSCA_E_INVALID, "unknown field");
    }
    if (bytes != need) return fail(sc, TURSCA_E_INVALID, "bytes does not match the field size");
    if (host) {
        CK(cudaStreamSynchronize(sc->st), "sync");
        CK(cudaMemcpy(dst, src, need, cudaMemcpyDefault), "get");
        return TURSCA_OK;
    }
    CK(cudaMemcpyAsync(dst, src, need, cudaMemcpyDefault, sc->st), "get");
    return sync_check(sc, "get");
}

long long tursca_launch_count(const tursca_scene *sc) { return sc ? sc->launches : 0; }

size_t tursca_scene_device_bytes(const tursca_scene *sc) {
    if (!sc) return 0;
    size_t b = sc->allocs.bytes;
    for (const DevBuf &v : sc->vbuf) b += v.cap;
    return b;
}

tursca_status tursca_set_option(tursca_scene *sc, int option, double value) {
    if (!sc) return fail(nullptr, TURSCA_E_INVALID, "scene is null");
    switch (option) {
        case TURSCA_OPT_RESIDUAL_FP64:
            sc->resid_fp64 = value != 0.0;
            return TURSCA_OK;
        case TURSCA_OPT_L2_RESIDENT: {
            if (value != 0.0 && value != 1.0) return fail(sc, TURSCA_E_INVALID, "L2 residency must be 0 or 1");
            if (value == 1.0) {
                // the set-aside of this context: as much of L2 as persisting lines may take
                int dev = 0;
                cudaDeviceProp prop;
                CK(cudaGetDevice(&dev), "device");
                CK(cudaGetDeviceProperties(&prop, dev), "device properties");
                size_t lim = 0;
                cudaDeviceGetLimit(&lim, cudaLimitPersistingL2CacheSize);
                if (prop.persistingL2CacheMaxSize > 0 && lim < (size_t)prop.persistingL2CacheMaxSize)
                    CK(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)prop.persistingL2CacheMaxSize),
                       "persisting L2 limit");
            }
            sc->l2_resident = (int)value;
            return TURSCA_OK;
        }
        case TURSCA_OPT_COUPLING_MIN:
            if (!(value >= 0.0) || !std::isfinite(value))
                return fail(sc, TURSCA_E_INVALID, "the coupling threshold must be finite and >= 0");
            if (value != sc->c_min) {
                sc->c_min = value;
                sc->assembled = sc->solved = sc->rendered = false;
            }
            return TURSCA_OK;
        case TURSCA_OPT_MAX_COUPLINGS:
            if (!(value >= 0.0) || value > 9.0e15 || value != std::floor(value))
                return fail(sc, TURSCA_E_INVALID, "the maximum number of couplings must be a whole number >= 0");
            if ((long long)value != sc->max_couplings) {
                sc->max_couplings = (long long)value;
                sc->assembled = sc->solved = sc->rendered = false;
            }
            return TURSCA_OK;
        case TURSCA_OPT_ANISO:
            if (value != 0.0 && value != 1.0 && value != 2.0)
                return fail(sc, TURSCA_E_INVALID, "anisotropic mode must be 0, 1 or 2");
            if ((int)value != sc->aniso) {
                sc->aniso = (int)value;
                sc->assembled = sc->solved = sc->rendered = false;
            }
            return TURSCA_OK;
        case TURSCA_OPT_SINGLE_SCATTER:
            if (value != 0.0 && value != 1.0) return fail(sc, TURSCA_E_INVALID, "single scatter must be 0 or 1");
            if ((int)value != sc->single) {
                sc->single = (int)value;
                sc->assembled = sc->solved = sc->rendered = false;
            }
            return TURSCA_OK;
        case TURSCA_OPT_GATHER_TILE:
            if (value != 0.0 && value != 1.0) return fail(sc, TURSCA_E_INVALID, "gather tile must be 0 or 1");
            sc->gather_tile = (int)value;
            return TURSCA_OK;
        case TURSCA_OPT_STAGE_VALUES:
            if (value != 0.0 && value != 1.0) return fail(sc, TURSCA_E_INVALID, "stage values must be 0 or 1");
            if (value == 1.0 && !sc->wq_auto && sc->wq == 6 && sc->d.precision != TURSCA_FP64)
                return fail(sc, TURSCA_E_INVALID, "the streamed passes take 4, 8 or 16 group warps");
            sc->stage_values = (int)value;
            if (sc->built && sc->wq_auto) sc->wq = tk::choose_wq(grid_c(sc), sc->d.precision == TURSCA_FP64);
            return TURSCA_OK;
        case TURSCA_OPT_GROUP_WARPS:
            if (value != 0.0 && value != 4.0 && value != 6.0 && value != 8.0 && value != 16.0)
                return fail(sc, TURSCA_E_INVALID, "group warps must be 0 (automatic), 4, 6, 8 or 16");
            if (value == 6.0 && sc->stage_values && sc->d.precision != TURSCA_FP64)
                return fail(sc, TURSCA_E_INVALID, "the streamed passes take 4, 8 or 16 group warps");
            sc->wq_auto = value == 0.0;
            if (value == 0.0) {
                if (sc->built) sc->wq = tk::choose_wq(grid_c(sc), sc->d.precision == TURSCA_FP64);
            } else {
                sc->wq = (int)value;
            }
            return TURSCA_OK;
        default: return fail(sc, TURSCA_E_INVALID, "unknown option");
    }
}

tursca_status tursca_profile_enable(tursca_scene *sc, int on) {
    if (!sc) return fail(nullptr, TURSCA_E_INVALID, "scene is null");
    CK(cudaStreamSynchronize(sc->st), "sync");
    sc->prof = on != 0;
    sc->ev_used = 0;
    return TURSCA_OK;
}

tursca_status tursca_profile_read(tursca_scene *sc, tursca_kernel_stat *out, int n, int *n_out) {
    if (!sc || !out || n < 0) return fail(sc, TURSCA_E_INVALID, "bad arguments");
    CK(cudaStreamSynchronize(sc->st), "sync");
    double ms[kNProf] = {};
    long long cnt[kNProf] = {};
    for (size_t i = 0; i < sc->ev_used; ++i) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, sc->ev[2 * i], sc->ev[2 * i + 1]), "event time");
        ms[sc->ev_cat[i]] += t;
        cnt[sc->ev_cat[i]] += sc->ev_n[i];
    }
    sc->ev_used = 0;
    int m = std::min(n, kNProf);
    for (int c = 0; c < m; ++c) {
        std::snprintf(out[c].name, sizeof(out[c].name), "%s", kProfNames[c]);
        out[c].launches = cnt[c];
        out[c].total_ms = ms[c];
    }
    if (n_out) *n_out = m;
    return TURSCA_OK;
}

tursca_status tursca_selftest_barrier(void *cuda_stream, int blocks, int arrive) {
    if (blocks < 1 || blocks > 1024) return fail(nullptr, TURSCA_E_INVALID, "blocks must be in 1..1024");
    const int r = tk::batch_barrier_selftest((cudaStream_t)cuda_stream, blocks, arrive);
    if (r < 0) return fail(nullptr, TURSCA_E_CUDA, "barrier self-test: CUDA error");
    return r ? TURSCA_E_TIMEOUT : TURSCA_OK;
}

tursca_status tursca_selftest_aniso_contract(tursca_scene *sc, int which, int tensor_cores, const void *X,
                                            void *out) {
    if (!sc) return fail(nullptr, TURSCA_E_INVALID, "scene is null");
    if (which != 0 && which != 1) return fail(sc, TURSCA_E_INVALID, "which must be 0 or 1");
    if (!out || (which == 0 && !X)) return fail(sc, TURSCA_E_INVALID, "null buffer");
    if (sc->d.precision == TURSCA_FP64) return fail(sc, TURSCA_E_UNSUPPORTED, "FP32 scenes only");
    if (!sc->assembled || !sc->aniso_asm) return fail(sc, TURSCA_E_STATE, "no anisotropic assembly");
    if (tensor_cores && which == 1)
        return fail(sc, TURSCA_E_UNSUPPORTED, "the routing denominators run on the CUDA cores only");
    if (tensor_cores && (!sc->ani_Bl || sc->aniso != 1))
        return fail(sc, TURSCA_E_STATE, "no tensor-core operands");
    tk::AniP<float> a = ani_p<float>(sc);
    a.mma = tensor_cores ? 1 : 0;
    const tk::GridC g = grid_c(sc);
    float *Xs = nullptr;
    if (which == 0) {  // X with the internal row stride, in the scene's X buffer
        Xs = (float *)sc->ani_X;
        CK(cudaMemcpy2DAsync(Xs, (size_t)a.ldx * sizeof(float), X, (size_t)g.n_nodes * sizeof(float),
                             (size_t)g.n_nodes * sizeof(float), (size_t)g.nd + g.ngd, cudaMemcpyDeviceToDevice, sc->st),
           "copy X");
    }
    CK(tk::launch_aniso_contract_test(sc->st, g, graph_p(sc), field_p<float>(sc), a, Xs, (float *)out, which,
                                      tensor_cores != 0),
       "contraction");
    CK(cudaGetLastError(), "contraction launch");
    return sync_check(sc, "contraction");
}

tursca_status tursca_selection_info(const tursca_scene *sc, double *threshold, long long *n_couplings,
                                    long long *n_kept) {
    if (!sc) return fail(nullptr, TURSCA_E_INVALID, "scene is null");
    if (!sc->assembled) return fail(const_cast<tursca_scene *>(sc), TURSCA_E_STATE, "no assembly yet");
    if (threshold) *threshold = sc->c_eff;
    if (n_couplings) *n_couplings = sc->n_couplings;
    if (n_kept) *n_kept = sc->n_kept;
    return TURSCA_OK;
}

tursca_status tursca_graph_info(const tursca_grid_desc *desc, tursca_graph_stats *out) {
    if (!out) return fail(nullptr, TURSCA_E_INVALID, "out is null");
    std::string m = check_desc(desc);
    if (!m.empty()) return fail(nullptr, TURSCA_E_INVALID, m);
    tg::Graph G;
    m = tg::build_graph(G, desc->nx, desc->ny, desc->nz, desc->hx, desc->hy, desc->hz, desc->stencil_radius,
                        desc->fib_points);
    if (!m.empty()) return fail(nullptr, TURSCA_E_INVALID, m);
    out->n_atm = G.n_atm;
    out->n_ground = G.n_ground;
    out->n_nodes = G.n_nodes;
    out->n_dirs = (int)G.dirs.size();
    out->n_up_dirs = (int)G.up_dirs.size();
    out->n_gdirs = (int)G.gdirs.size();
    out->n_gmembers = G.n_gmembers;
    out->nnz = G.nnz;
    out->nnz_edges = G.nnz_edges;
    out->n_classes = (int)G.classes.size();
    out->max_row = G.max_row;
    return TURSCA_OK;
}

tursca_status tursca_graph_structure(const tursca_grid_desc *desc, int32_t *row_ptr, int32_t *col, int16_t *dir,
                                     int8_t *k) {
    std::string m = check_desc(desc);
    if (!m.empty()) return fail(nullptr, TURSCA_E_INVALID, m);
    tg::Graph G;
    m = tg::build_graph(G, desc->nx, desc->ny, desc->nz, desc->hx, desc->hy, desc->hz, desc->stencil_radius,
                        desc->fib_points);
    if (!m.empty()) return fail(nullptr, TURSCA_E_INVALID, m);
    tg::expand_csr(G, row_ptr, col, dir, k);
    return TURSCA_OK;
}

tursca_status tursca_quadrature(const tursca_grid_desc *desc, double *q_iso, double *q_lamb) {
    std::string m = check_desc(desc);
    if (!m.empty()) return fail(nullptr, TURSCA_E_INVALID, m);
    tg::Graph G;
    m = tg::build_graph(G, desc->nx, desc->ny, desc->nz, desc->hx, desc->hy, desc->hz, desc->stencil_radius,
                        desc->fib_points);
    if (!m.empty()) return fail(nullptr, TURSCA_E_INVALID, m);
    if (q_iso) std::memcpy(q_iso, G.q_iso.data(), G.q_iso.size() * sizeof(double));
    if (q_lamb) std::memcpy(q_lamb, G.q_lamb.data(), G.q_lamb.size() * sizeof(double));
    return TURSCA_OK;
}

const char *tursca_status_string(tursca_status s) {
    switch (s) {
        case TURSCA_OK: return "ok";
        case TURSCA_E_INVALID: return "invalid argument";
        case TURSCA_E_NOMEM: return "out of memory";
        case TURSCA_E_CUDA: return "CUDA error";
        case TURSCA_E_NOT_CONVERGED: return "solver did not converge";
        case TURSCA_E_TIMEOUT: return "device wait timed out";
        case TURSCA_E_STATE: return "call out of order";
        case TURSCA_E_UNSUPPORTED: return "not available";
    }
    return "unknown status";
}

tursca_status tursca_last_error(const tursca_scene *sc, char *buf, size_t n) {
    if (!buf || n == 0) return TURSCA_E_INVALID;
    const std::string &m = sc ? sc->err : g_last_error;
    std::snprintf(buf, n, "%s", m.c_str());
    return TURSCA_OK;
}

}  // extern "C"

namespace tk {
void scene_attach_batcher(tursca_scene *sc, ChebBatcher *b) {
    if (!sc || sc->d.precision == TURSCA_FP64) return;
    if (b && !sc->bready) {
        if (cudaEventCreateWithFlags(&sc->bready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sc->bdone, cudaEventDisableTiming) != cudaSuccess)
            return;
    }
    sc->batcher = b;
}
}  // namespace tk

