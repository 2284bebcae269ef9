// api.cu -- the extern "C" entry points of libedp.so (see include/edp.h):
// argument validation, workspace layout, launch configuration and the pass
// schedule of Algorithm 1.
#include <algorithm>
#include <climits>
#include <cstring>

#include "edp.h"
#include "kernels.h"

using namespace edp;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kHeader = 256;  // status word + reserved
constexpr int kMaxSmem = 227 * 1024;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int g_tune_rb = 0;       // rows per block override (0 = automatic)
int g_tune_e = 0;        // labels per lane target override, scanline DP (0 = automatic)
int g_tune_t = 0;        // warps per row override, multi-axis scan pass (0 = automatic)
int g_force_general = 0; // 1: one-axis problems also take the multi-axis pass kernel
int g_generic_team = 0;  // 1: multi-axis problems take the generic team body (tests)
int g_line_mode = 0;     // two-axis line kernel: 0 where it is faster (65-label lines), 1 off, 2 wherever built
int g_line_split = 1;    // 65 x 65 labels: lines split over lane pairs (0: one lane per line)
int g_fused_cost = 0;    // edp_solve_images: the split line kernel computes the pair cost from the images
int g_pass_pairs = 2;    // P1 + P2 and P3 + P4 as paired sweeps: 0 never, 1 always, 2 when every band is resident
int g_last_launches = 0; // scan-pass launches of the most recent solve
const char *g_last_kernel = "";  // scan-pass kernel of the most recent solve
constexpr long long kSpinDefault = 4000000;
long long g_spin_limit = kSpinDefault;  // polls before an inter-block wait gives up
int g_hold_band = 0;     // test hook: the band whose first row waits for records never written
int g_batch_alone_pixels = 172800;  // batched solve: problems of this many pixels or more get their own launches
void *const *g_prof_events = nullptr;  // optional per-pass events (profiling hook)
int g_prof_n = 0;
unsigned long long *g_trace = nullptr;  // optional per-band trace buffer (device)
size_t g_trace_bytes = 0;

struct Geometry {
    int R;       // label axes after dropping axes with one label
    int Qr[3];   // their sizes
    int Q;       // total labels
};

// Validation shared by every entry point.  Axes with a single label carry no
// prior term and are dropped for the DP kernels (the linear label index is
// unchanged by that).
int check_space(const edp_label_space *s, Geometry *g) {
    if (!s) return EDP_ERR_INVALID_ARG;
    if (s->R < 1 || s->R > 3) return EDP_ERR_INVALID_ARG;
    long long Q = 1;
    g->R = 0;
    for (int r = 0; r < 3; ++r) {
        if (s->Q[r] < 1) return EDP_ERR_INVALID_ARG;
        if (r >= s->R && s->Q[r] != 1) return EDP_ERR_INVALID_ARG;
        if (r < s->R && s->step[r] != 1 && s->step[r] != -1) return EDP_ERR_INVALID_ARG;
        Q *= s->Q[r];
        if (s->Q[r] > 1) g->Qr[g->R++] = s->Q[r];
    }
    if (Q > (1 << 20)) return EDP_ERR_UNSUPPORTED;
    if (g->R == 0) {
        g->R = 1;
        g->Qr[0] = 1;
    }
    for (int r = g->R; r < 3; ++r) g->Qr[r] = 1;
    g->Q = (int)Q;
    return EDP_OK;
}

int check_prior(const edp_params *p) {
    if (!p) return EDP_ERR_INVALID_ARG;
    if (p->lambda < 0 || p->g < 1 || p->cmax < 0) return EDP_ERR_INVALID_ARG;
    if (p->l1 != 1 && p->l1 != 2) return EDP_ERR_INVALID_ARG;
    if (p->prior_mode != EDP_PRIOR_JOINT && p->prior_mode != EDP_PRIOR_PER_AXIS) return EDP_ERR_INVALID_ARG;
    return EDP_OK;
}

long long cap_value(const edp_params *p) {
    const long long gg = p->l1 == 1 ? p->g : (long long)p->g * p->g;
    return (long long)p->lambda * gg;
}

int pow2ceil(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Lanes per line G and labels per lane E for a line of L labels.
bool choose_axis(int L, int etarget, AxisCfg *a) {
    int G = pow2ceil((L + etarget - 1) / etarget);
    if (G > 32) G = 32;
    int E = (L + G - 1) / G;
    if (E > kEM) return false;
    a->L = L;
    a->G = G;
    a->E = E;
    return true;
}

int em_for(int E) {
    if (E <= 2) return 2;
    if (E <= 4) return 4;
    if (E <= 8) return 8;
    return 16;
}

struct DpConfig {
    AxisCfg ax[3];
    int em;
    int RB;
    int threads;
    size_t smem;
};

// smem bytes of one EDP pass block / scanline block
size_t pass_smem(int RB, int Q, int R) {
    // argk, gmin, msgA, ringB[2], staging[2][3], tmpA/tmpB (R >= 2)
    return (size_t)RB * 2 * 8 + (size_t)RB * 4 * 4 + (size_t)RB * Q * 4 * (R >= 2 ? 11 : 9);
}
size_t scan_smem(int RB, int Q, int R, int W, int ptr_bytes, bool ptr_smem) {
    // gkey, tmpk (R >= 2), S, staging[2]
    size_t s = (size_t)RB * 2 * 8 + (size_t)RB * Q * (R >= 2 ? 8 : 0) + (size_t)RB * Q * 4 * 3;
    if (ptr_smem) s += (size_t)RB * W * Q * ptr_bytes;
    return s;
}

int configure(const Geometry &g, int H, bool scan, int W, int ptr_bytes, bool *ptr_smem, DpConfig *c) {
    const int etarget = g_tune_e > 0 ? g_tune_e : (g.R == 1 ? 4 : 5);
    int stride = 1;
    int maxE = 1;
    for (int r = 0; r < g.R; ++r) {
        if (g.Qr[r] > kMaxLine) return EDP_ERR_UNSUPPORTED;
        if (!choose_axis(g.Qr[r], etarget, &c->ax[r])) return EDP_ERR_UNSUPPORTED;
        c->ax[r].nlines = g.Q / g.Qr[r];
        c->ax[r].stride = stride;
        stride *= g.Qr[r];
        maxE = std::max(maxE, c->ax[r].E);
    }
    for (int r = g.R; r < 3; ++r) c->ax[r] = AxisCfg{1, 1, 1, g.Q, stride};
    c->em = em_for(maxE);
    const int gpw0 = 32 / c->ax[0].G;
    auto threads_for = [&](int RB) { return ((RB * c->ax[0].nlines + gpw0 - 1) / gpw0) * 32; };
    int RB;
    if (g_tune_rb > 0) {
        RB = g_tune_rb;
    } else {
        const int per_row = threads_for(1);
        RB = std::max(1, 256 / per_row);
    }
    RB = std::min(RB, H);
    RB = std::max(RB, 1);
    bool psm = false;
    if (scan) {
        psm = scan_smem(RB, g.Q, g.R, W, ptr_bytes, true) <= (size_t)kMaxSmem / 2;
        while (RB > 1 && scan_smem(RB, g.Q, g.R, W, ptr_bytes, psm) > (size_t)kMaxSmem) --RB;
        c->smem = scan_smem(RB, g.Q, g.R, W, ptr_bytes, psm);
    } else {
        while (RB > 1 && pass_smem(RB, g.Q, g.R) > (size_t)kMaxSmem) --RB;
        c->smem = pass_smem(RB, g.Q, g.R);
    }
    if (c->smem > (size_t)kMaxSmem) return EDP_ERR_UNSUPPORTED;
    c->RB = RB;
    c->threads = std::min(kMaxThreads, std::max(32, threads_for(RB)));
    if (ptr_smem) *ptr_smem = psm;
    return EDP_OK;
}

int ptr_bytes_for(int Q) { return Q <= 256 ? 1 : (Q <= 65536 ? 2 : 4); }

// Workspace of edp_solve:
//   header | consumed columns [4*iters][H] | band counters [4*iters] |
//   hand-off records | M[4][N*Qm]
// Messages are stored with the vector stride Qm = Q rounded up to a multiple
// of 4 (16-byte aligned pixel vectors).  The hand-off records are sized for
// both scan-pass kernels: {value, tag} per label of the last row of each row
// band -- one-axis kernel: every column, bands of kMinRowsR1 rows; multi-axis
// kernel: a ring of team_ring(W) columns, bands of one row or more.
constexpr int kMinRowsR1 = 2;
constexpr int kResidentMin = 128;  // resident blocks assumed when sizing the record ring
constexpr int kLineRingResident = 4;  // record ring columns of the line kernel when every band is resident
int msg_stride(int Q) { return (Q + 3) / 4 * 4; }
// columns of the record ring: the first of K resident bands may run
// (K - 1) * ring columns ahead of the last, which must cover the row
int team_ring(int W, int resident) { return std::max(8, (W + resident - 2) / std::max(1, resident - 1) + 2); }
struct SolveLayout {
    size_t cons, counters, lcons, lflag, ll, ll_bytes, msg[4], end;
    int Qm;
};
SolveLayout solve_layout(int W, int H, int Q, int R, int iters) {
    SolveLayout L;
    const size_t npass = 4 * (size_t)iters;
    L.Qm = msg_stride(Q);
    L.cons = kHeader;
    L.counters = align_up(L.cons + npass * H * 4);
    // two-axis line kernels: per-warp consumed columns and producer flags of
    // the record ring, [4*iters][H][kLineFlagStride] each
    L.lcons = align_up(L.counters + npass * 4);
    L.lflag = align_up(L.lcons + npass * H * kLineFlagStride * 4);
    L.ll = align_up(L.lflag + npass * H * kLineFlagStride * 4);
    // one-axis kernel: a record per column of a paired sweep (2W) for every band boundary
    const size_t r1 = (R == 1 && Q <= 256) ? (size_t)((H + kMinRowsR1 - 1) / kMinRowsR1) * 2 * W * Q * 8 : 0;
    const size_t tm = (size_t)H * team_ring(2 * W, kResidentMin) * L.Qm * 8;  // paired sweeps: 2W columns
    L.ll_bytes = std::max(r1, tm);
    size_t off = align_up(L.ll + L.ll_bytes);
    for (int k = 0; k < 4; ++k) {
        L.msg[k] = off;
        off = align_up(off + (size_t)W * H * L.Qm * 4);
    }
    L.end = off;
    return L;
}

struct ImagesLayout {
    SolveLayout s;
    size_t C, img[3], labels, energy, end;
};
ImagesLayout images_layout(int W, int H, int Q, int R, int iters) {
    ImagesLayout L;
    L.s = solve_layout(W, H, Q, R, iters);
    L.C = L.s.end;
    size_t off = align_up(L.C + (size_t)W * H * Q * 4);
    for (int k = 0; k < 3; ++k) {
        L.img[k] = off;
        off = align_up(off + (size_t)W * H);
    }
    L.labels = off;
    off = align_up(off + (size_t)W * H * 4);
    L.energy = off;
    L.end = align_up(off + 4 * 8);
    return L;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? EDP_OK : EDP_ERR_CUDA; }

int check_range(int W, int H, const Geometry &g, const edp_params *p) {
    const long long N = (long long)W * H;
    if (p->lambda > (1 << 20)) return EDP_ERR_RANGE;
    if (cap_value(p) * g.R > (1 << 28)) return EDP_ERR_RANGE;
    const long long bound = N * (p->cmax + 2LL * g.R * cap_value(p)) * 2;
    if (bound >= (1LL << 31)) return EDP_ERR_RANGE;
    return EDP_OK;
}

// Multi-axis kernel shape: warps per row (team), per-axis lane groups.
// Cost model of one column step: every round of an axis runs the two
// in-lane sweeps over E labels; lane groups add the carry exchange.
struct TeamShape {
    int T, em;
    TeamAxis ax[3];
    long cost;
};
bool team_shape(const Geometry &g, int T, int gpar, TeamShape *S) {
    const int NL = 32 * T;
    int stride = 1, maxE = 1;
    S->T = T;
    S->cost = (g.R > 1 && T > 1 ? 24L * g.R : 0) + 10L * T;  // barriers, per-warp overhead
    for (int r = 0; r < g.R; ++r) {
        const int L = g.Qr[r], nlines = g.Q / L;
        long best = -1;
        TeamAxis bx{};
        for (int G = 1; G <= 32; G <<= 1) {
            const int E = (L + G - 1) / G;
            if (E > 33) continue;
            if (G > 1 && (L + G / 2 - 1) / (G / 2) <= 1) break;  // more lanes than labels
            const int rounds = (int)(((long)nlines * G + NL - 1) / NL);
            const int kc = (G > 1 && gpar > 1) ? std::min(G - 1, (gpar - 1 + E - 1) / E) : 0;
            int lg = 0;
            while ((1 << lg) < G) ++lg;
            const long c = (long)rounds * (5L * E + (G > 1 ? 4L * E + 10L * kc + 6L * lg : 0) + 12);
            if (best < 0 || c < best) {
                best = c;
                bx = TeamAxis{L, G, E, nlines, stride, kc, rounds};
            }
        }
        if (best < 0) return false;
        S->ax[r] = bx;
        S->cost += best;
        maxE = std::max(maxE, bx.E);
        stride *= L;
    }
    for (int r = g.R; r < 3; ++r) S->ax[r] = TeamAxis{1, 1, 1, g.Q, stride, 0, 0};
    S->em = maxE <= 9 ? 9 : (maxE <= 17 ? 17 : 33);
    return true;
}

// Everything about one EDP problem that does not change from pass to pass:
// which band body runs it, the launch shape and the argument blocks.
// max_threads / fixed_threads: block size limit, or the block size of a
// batched launch (0 = free).
struct SolvePlan {
    bool r1;          // warp-per-row body (one label axis, Q <= 256)
    bool line;        // two-axis line kernel (one label line per lane)
    bool split;       // its form with each line split over two lanes
    int Q0, Q1;       // its label-space shape
    int nbands;
    int threads;
    int em;
    int laps;         // record ring laps per pass (multi-axis kernel)
    size_t smem;
    SolveLayout L;
    PassR1Args o;
    TeamArgs ta;
};

int plan_solve(const int32_t *C, int W, int H, const Geometry &g, const edp_params *p, int32_t *labels,
               unsigned char *ws, SolvePlan *P, int fixed_threads = 0) {
    memset(P, 0, sizeof *P);
    P->L = solve_layout(W, H, g.Q, g.R, p->iters);
    const SolveLayout &L = P->L;
    int *M[4];
    for (int k = 0; k < 4; ++k) M[k] = reinterpret_cast<int *>(ws + L.msg[k]);
    P->r1 = (g.R == 1 && g.Q <= 256 && !g_force_general);
    if (P->r1) {
        const int E = (g.Q + 31) / 32;
        int NWR = fixed_threads ? fixed_threads / 32 : (g_tune_rb > 0 ? g_tune_rb : 8);
        if (!fixed_threads) NWR = std::max(kMinRowsR1, std::min(NWR, std::min(pass_r1_max_rows(E, p->l1), H)));
        while (!fixed_threads && NWR > kMinRowsR1 && pass_r1_smem(NWR, E) > (size_t)kMaxSmem) --NWR;
        P->smem = pass_r1_smem(NWR, E);
        if (P->smem > (size_t)kMaxSmem) return EDP_ERR_UNSUPPORTED;
        PassR1Args &a = P->o;
        a.C = C;
        for (int k = 0; k < 4; ++k) a.M[k] = M[k];
        a.labels = labels;
        a.ll = reinterpret_cast<int2 *>(ws + L.ll);
        a.status = reinterpret_cast<int *>(ws);
        a.W = W;
        a.H = H;
        a.Q = g.Q;
        a.Qm = L.Qm;
        a.E = E;
        a.EMt = E;
        // widest prefetch copy that divides E and Q and keeps 4*vw-byte alignment
        a.vw = 1;
        for (int v : {4, 2}) {
            const uintptr_t al = 4 * v;
            bool ok = E % v == 0 && g.Q % v == 0 && reinterpret_cast<uintptr_t>(C) % al == 0;
            for (int k = 0; k < 4; ++k) ok = ok && reinterpret_cast<uintptr_t>(M[k]) % al == 0;
            if (ok) {
                a.vw = v;
                break;
            }
        }
        a.lam = p->lambda;
        a.capv = (int)cap_value(p);
        a.kc = p->g <= 1 ? 0 : std::min(31, (p->g - 1 + E - 1) / E);
        a.l1 = p->l1;
        a.g = p->g;
        a.NWR = NWR;
        a.nbands = (H + NWR - 1) / NWR;
        a.grid = a.nbands;
        a.spin_limit = g_spin_limit;
        P->nbands = a.nbands;
        P->threads = 32 * NWR;
        P->em = a.EMt;
        return EDP_OK;
    }
    // two label axes with a build of the line kernel (one label line per
    // lane): single-problem solves of the linear prior
    // (measured: faster than the whole-line multi-axis form where lines hold
    // 65 labels, whose rows the multi-axis kernel cannot all keep resident;
    // slower at 33 x 33)
    // The quadratic prior: the line kernel serves the shapes it has a build
    // for (no other form serves them with l1 = 2).
    const bool line_pick = g_line_mode == 2 ||
                           (g_line_mode == 0 && (std::max(g.Qr[0], g.Qr[1]) > 33 || p->l1 == 2));
    if (!fixed_threads && g.R == 2 && line_pick && !g_generic_team && pass_line_built(g.Qr[0], g.Qr[1], p->l1)) {
        P->line = true;
        P->Q0 = g.Qr[0];
        P->Q1 = g.Qr[1];
        // lines split over lane pairs where built; the completions of the
        // split sweeps add up to 33 lambda, bounded here for the heaviest
        // per-edge multiplier (255)
        P->split = g_line_split && pass_line_split_built(P->Q0, P->Q1, p->l1) &&
                   (long long)p->lambda * 255 <= pass_line_split_max_lambda();
        const bool split = P->split;
        const int TW = pass_line_warps(P->Q0, P->Q1, split);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        sms = std::max(1, sms);
        // rows per block: every row band resident, the fewest rows on the
        // busiest SM (blocks are spread evenly), then the most rows per block
        // (fewer hand-offs between blocks); one row per block when no shape
        // keeps every band resident
        int NT = 1;
        if (g_tune_rb > 0) {
            NT = std::min(g_tune_rb, 4);
        } else {
            int best = INT_MAX;
            for (int nt = 1; nt <= 4; ++nt) {
                const int nb = (H + nt - 1) / nt;
                const size_t sm = pass_line_smem(nt, P->Q0, P->Q1, split);
                if (sm > (size_t)kMaxSmem) break;
                const int occ = edp_pass_line_occupancy(P->Q0, P->Q1, p->l1, split, 32 * TW * nt, sm);
                if (occ < 1 || nb > occ * sms) continue;
                const int load = nt * ((nb + sms - 1) / sms);
                if (load <= best) {
                    best = load;
                    NT = nt;
                }
            }
        }
        NT = std::max(1, std::min(NT, H));
        P->smem = pass_line_smem(NT, P->Q0, P->Q1, split);
        if (P->smem > (size_t)kMaxSmem) return EDP_ERR_UNSUPPORTED;
        TeamArgs &a = P->ta;
        a.C = C;
        for (int k = 0; k < 4; ++k) a.M[k] = M[k];
        a.labels = labels;
        a.ll = reinterpret_cast<int2 *>(ws + L.ll);
        a.status = reinterpret_cast<int *>(ws);
        a.W = W;
        a.H = H;
        a.Q = g.Q;
        a.Qm = L.Qm;
        a.R = g.R;
        a.lam = p->lambda;
        a.capv = (int)cap_value(p);
        a.mode = p->prior_mode;
        a.l1 = p->l1;
        a.g = p->g;
        a.T = TW;
        a.NT = NT;
        a.nbands = (H + NT - 1) / NT;
        // record ring: when every band is resident, consecutive bands run about
        // one column apart, so a short ring suffices and stays in L2; otherwise
        // the depth that lets the first resident band finish its row
        {
            const int occ = edp_pass_line_occupancy(P->Q0, P->Q1, p->l1, split, 32 * TW * NT, P->smem);
            const bool all_resident = a.nbands <= std::max(1, occ) * sms;
            a.ring = all_resident ? std::min(kLineRingResident, team_ring(2 * W, kResidentMin))
                                  : team_ring(2 * W, kResidentMin);
        }
        a.spin_limit = g_spin_limit;
        P->laps = (2 * W + a.ring - 1) / a.ring;
        P->nbands = a.nbands;
        P->threads = 32 * TW * NT;
        P->em = 0;
        return EDP_OK;
    }
    // multi-axis (team) kernel.  Lean form: two or more axes whose lines hold
    // 9, 17 or 33 labels (or all 65), Tv warps per message vector, lanes
    // owning whole lines.
    TeamShape S;
    bool lean = g.R >= 2 && !g_generic_team;
    int LM = 0, Tv = 0;
    bool short_lines = true, all65 = true;
    for (int r = 0; r < g.R; ++r) {
        LM = std::max(LM, g.Qr[r]);
        short_lines = short_lines && (g.Qr[r] == 9 || g.Qr[r] == 17 || g.Qr[r] == 33);
        all65 = all65 && g.Qr[r] == 65;
    }
    // 65-label lines: a build of their own (single-problem kernel only; the
    // quadratic-prior build serves every line length of the form)
    lean = lean && (short_lines || (all65 && (!fixed_threads || p->l1 == 2)));
    const int tmax = fixed_threads ? std::min(12, fixed_threads / 32) : (lean ? 8 : 12);
    if (lean) {
        LM = p->l1 == 2 ? 2 : (all65 ? 65 : 33);
        int maxlines = 1;
        for (int r = 0; r < g.R; ++r) maxlines = std::max(maxlines, g.Q / g.Qr[r]);
        // one lane per line and vector; 65-label lines (many labels per line,
        // HBM-heavy) run best with the widest team (measured)
        Tv = g_tune_t > 0 ? std::max(1, g_tune_t / 2) : std::min(maxlines > 64 ? 4 : (maxlines + 31) / 32, 4);
        if (2 * Tv > tmax) Tv = tmax / 2;
        if (Tv < 1) return EDP_ERR_UNSUPPORTED;
        S.T = 2 * Tv;
        S.em = LM;
        int stride = 1;
        for (int r = 0; r < 3; ++r) {
            const int L = r < g.R ? g.Qr[r] : 1;
            S.ax[r] = TeamAxis{L, 1, L, g.Q / L, stride, 0, 1};
            stride *= L;
        }
    } else {
        if (p->l1 != 1) return EDP_ERR_UNSUPPORTED;  // quadratic taps: one-axis, lean and windowed forms
        bool have = false;
        if (g_tune_t > 0) {
            if (g_tune_t > tmax || !team_shape(g, g_tune_t, p->g, &S)) return EDP_ERR_UNSUPPORTED;
            if (S.em > 17 && S.T > 8) return EDP_ERR_UNSUPPORTED;
            have = true;
        } else {
            for (int T = 1; T <= tmax; ++T) {
                if (g.R == 1 && T > 1) break;  // one line: one warp
                TeamShape c;
                if (!team_shape(g, T, p->g, &c)) continue;
                if (c.em > 17 && T > 8) continue;  // built for <= 256 threads (<= 384 otherwise)
                if (!have || c.cost * 10 < S.cost * 9) {
                    S = c;
                    have = true;
                }
            }
        }
        if (!have) return EDP_ERR_UNSUPPORTED;
    }
    const int T = S.T;
    const int thr_cap = fixed_threads ? fixed_threads : (lean || S.em > 17 ? 256 : 384);
    int NT = 0, nbuf = 3, kmb = 4;
    for (int attempt = 0; attempt < 3 && NT < 1; ++attempt) {
        if (attempt == 1) nbuf = kmb = 2;
        if (attempt == 2) kmb = 1;  // one team per block: the slot of the copied-in records only
        NT = std::min(thr_cap / (32 * T), attempt == 2 ? 1 : 15);
        while (NT > 0 && pass_team_smem(NT, L.Qm, g.R, nbuf, kmb) > (size_t)kMaxSmem) --NT;
    }
    if (NT < 1) return EDP_ERR_UNSUPPORTED;
    if (!fixed_threads) {
        int want = g_tune_rb > 0 ? g_tune_rb : 4;
        while (g_tune_rb <= 0 && want > 1 && (H + want - 1) / want < 100) --want;
        NT = std::max(1, std::min(NT, want));
    }
    NT = std::min(NT, H);
    if (kmb == 1 && NT > 1) return EDP_ERR_UNSUPPORTED;
    TeamArgs &a = P->ta;
    a.C = C;
    for (int k = 0; k < 4; ++k) a.M[k] = M[k];
    a.labels = labels;
    a.ll = reinterpret_cast<int2 *>(ws + L.ll);
    a.status = reinterpret_cast<int *>(ws);
    a.W = W;
    a.H = H;
    a.Q = g.Q;
    a.Qm = L.Qm;
    a.R = g.R;
    for (int r = 0; r < 3; ++r) a.ax[r] = S.ax[r];
    a.lam = p->lambda;
    a.capv = (int)cap_value(p);
    a.mode = p->prior_mode;
    a.T = T;
    a.NT = NT;
    a.nbuf = nbuf;
    a.kmb = kmb;
    a.ring = team_ring(2 * W, kResidentMin);
    a.em = S.em;
    a.lean = lean;
    a.l1 = p->l1;
    a.g = p->g;
    a.nbands = (H + NT - 1) / NT;
    a.spin_limit = g_spin_limit;
    P->laps = (W + a.ring - 1) / a.ring;
    P->nbands = a.nbands;
    P->threads = fixed_threads ? fixed_threads : 32 * T * NT;
    P->em = S.em;
    P->smem = pass_team_smem(NT, L.Qm, g.R, nbuf, kmb);
    return EDP_OK;
}

// Control words that must start from zero before the first pass: status,
// consumed-column and band counters, and the used hand-off records.
size_t control_bytes(const SolvePlan &P, int W, int Q) {
    return P.r1 ? P.L.ll + (size_t)P.nbands * 2 * W * Q * 8 : P.L.ll + (size_t)P.nbands * P.ta.ring * P.L.Qm * 8;
}

bool pairs_for(bool resident) { return g_pass_pairs == 1 || (g_pass_pairs == 2 && resident); }

// Launch k of iteration `it`: one pass (k = 0..3), or with paired sweeps the
// pair k = 0 (P1 + P2) or 1 (P3 + P4).  Sets the first pass and the flags of
// both passes of the launch.
template <typename Args>
int set_launch(Args &a, int it, int k, int iters, bool pairs) {
    const int pass = pairs ? 2 * k : k;
    const PassFlags f = pass_flags(it, pass, iters);
    const PassFlags f2 = pass_flags(it, pairs ? pass + 1 : pass, iters);
    a.pass = pass;
    a.read_c = f.read_c;
    a.read_d = f.read_d;
    a.write_a = f.write_a;
    a.write_b = f.write_b;
    a.final_ = f.final_;
    a.pair = pairs;
    a.read_c2 = f2.read_c;
    a.write_a2 = f2.write_a;
    a.write_b2 = f2.write_b;
    a.final2 = f2.final_;
    return pass;
}

// The pair cost (Eq. Cost_value) as the split line kernel and the energy
// kernel compute it from the images, in place of a cost volume.
struct FusedImages {
    const uint8_t *I0, *I1;
    int pitch, v0, v1, t0, t1, cmax, l2;
};
FusedImages fused_images(const uint8_t *I0, const uint8_t *I1, int pitch, const edp_label_space *s,
                         const edp_params *p) {
    FusedImages f;
    f.I0 = I0;
    f.I1 = I1;
    f.pitch = pitch;
    f.v0 = s->vmin[0];
    f.v1 = s->R >= 2 ? s->vmin[1] : 0;
    f.t0 = s->step[0];
    f.t1 = s->R >= 2 ? s->step[1] : 0;
    f.cmax = p->cmax;
    f.l2 = p->l2;
    return f;
}

// wh / wv: optional per-edge prior multipliers (one-axis kernel only);
// fi: the split line kernel computes the pair cost from these images (C is
// not read); the caller checks that the plan is that kernel
int run_solve(const int32_t *C, int W, int H, const Geometry &g, const edp_params *p, int32_t *labels,
              unsigned char *ws, cudaStream_t st, const uint8_t *wh = nullptr, const uint8_t *wv = nullptr,
              const FusedImages *fi = nullptr) {
    SolvePlan P;
    int rc = plan_solve(C, W, H, g, p, labels, ws, &P);
    if (rc) return rc;
    if (fi) {
        if (!P.line || !P.split) return EDP_ERR_UNSUPPORTED;
        P.ta.fI0 = fi->I0;
        P.ta.fI1 = fi->I1;
        P.ta.fpitch = fi->pitch;
        P.ta.fv0 = fi->v0;
        P.ta.fv1 = fi->v1;
        P.ta.ft0 = fi->t0;
        P.ta.ft1 = fi->t1;
        P.ta.fcmax = fi->cmax;
        P.ta.fl2 = fi->l2;
    }
    if (wh && !P.r1 && !P.line && !P.ta.lean) return EDP_ERR_UNSUPPORTED;  // not the lane-group form
    P.o.wh = P.ta.wh = wh;
    P.o.wv = P.ta.wv = wv;
    if ((rc = cuda_status(cudaMemsetAsync(ws, 0, control_bytes(P, W, g.Q), st)))) return rc;
    int grid_t = 1, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    bool resident;  // every row band has a block at once
    if (P.line) {
        const int occ = std::max(1, edp_pass_line_occupancy(P.Q0, P.Q1, P.ta.l1, P.split, P.threads, P.smem));
        grid_t = std::min(P.nbands, occ * sms);
        if (grid_t < P.nbands && team_ring(2 * W, grid_t) > P.ta.ring) return EDP_ERR_UNSUPPORTED;
        resident = grid_t >= P.nbands;
    } else if (!P.r1) {
        const int occ = std::max(1, edp_pass_team_occupancy(P.em, P.ta.lean, 0, P.threads, P.smem));
        grid_t = std::min(P.nbands, occ * sms);
        // a smaller resident set than the ring was sized for could stall the back-pressure
        if (grid_t < P.nbands && team_ring(2 * W, grid_t) > P.ta.ring) return EDP_ERR_UNSUPPORTED;
        resident = grid_t >= P.nbands;
    } else {
        resident = P.nbands <= std::max(1, edp_pass_r1_occupancy(P.o.E, P.o.l1, P.threads, P.smem)) * sms;
    }
    // paired sweeps: two launches per iteration (P1 + P2, P3 + P4).  They
    // shorten the wavefront when every band runs at once; when bands wait for
    // a free block, a paired band holds its block twice as long.
    const bool pairs = pairs_for(resident);
    const int per_it = pairs ? 2 : 4;
    g_last_launches = per_it * p->iters;
    g_last_kernel = P.r1     ? "edp_pass_r1_kernel"
                    : P.line ? (P.split ? "edp_pass_line2_kernel" : "edp_pass_line_kernel")
                             : "edp_pass_team_kernel";
    for (int it = 0; it < p->iters; ++it) {
        for (int k = 0; k < per_it; ++k) {
            const int launch = it * per_it + k;
            unsigned long long *trace = (g_trace && (size_t)(launch + 1) * P.nbands * 32 <= g_trace_bytes)
                                            ? g_trace + (size_t)launch * P.nbands * 4
                                            : nullptr;
            const bool prof = g_prof_events && 2 * launch + 1 < g_prof_n;
            if (prof && cudaEventRecord((cudaEvent_t)g_prof_events[2 * launch], st) != cudaSuccess)
                return EDP_ERR_CUDA;
            if (P.line) {
                TeamArgs a = P.ta;
                const int slot = it * 4 + set_launch(a, it, k, p->iters, pairs);
                a.cons = reinterpret_cast<unsigned *>(ws + P.L.lcons) + (size_t)slot * H * kLineFlagStride;
                a.rflag = reinterpret_cast<unsigned *>(ws + P.L.lflag) + (size_t)slot * H * kLineFlagStride;
                a.tag0 = 1 + slot * P.laps;
                a.hold_band = g_hold_band;
                a.band_counter = reinterpret_cast<unsigned *>(ws + P.L.counters) + slot;
                a.grid = grid_t;
                a.trace = trace;
                if (launch_edp_pass_line(a, P.Q0, P.Q1, P.split, P.threads, P.smem, st)) return EDP_ERR_CUDA;
            } else if (P.r1) {
                PassR1Args a = P.o;
                const int slot = it * 4 + set_launch(a, it, k, p->iters, pairs);  // counters of the first pass
                a.tag = slot + 1;
                a.hold_band = g_hold_band;
                a.band_counter = reinterpret_cast<unsigned *>(ws + P.L.counters) + slot;
                a.trace = trace;
                if (launch_edp_pass_r1(a, P.threads, P.smem, st)) return EDP_ERR_CUDA;
            } else {
                TeamArgs a = P.ta;
                // a pair takes the record tags of both its passes' slots
                const int slot = it * 4 + set_launch(a, it, k, p->iters, pairs);
                a.cons = reinterpret_cast<unsigned *>(ws + P.L.cons) + (size_t)slot * H;
                a.tag0 = 1 + slot * P.laps;
                a.hold_band = g_hold_band;
                a.band_counter = reinterpret_cast<unsigned *>(ws + P.L.counters) + slot;
                a.grid = grid_t;
                a.trace = trace;
                if (launch_edp_pass_team(a, P.threads, P.smem, st)) return EDP_ERR_CUDA;
            }
            if (prof && cudaEventRecord((cudaEvent_t)g_prof_events[2 * launch + 1], st) != cudaSuccess)
                return EDP_ERR_CUDA;
        }
    }
    return EDP_OK;
}

int check_images(const uint8_t *I0, const uint8_t *I1, const uint8_t *I2, int W, int H, int pitch,
                 const edp_label_space *s, const edp_params *p) {
    if (!I0 || !I1 || W < 1 || H < 1 || pitch < W) return EDP_ERR_INVALID_ARG;
    if (!s || !p) return EDP_ERR_INVALID_ARG;
    if (p->l2 != 1 && p->l2 != 2) return EDP_ERR_INVALID_ARG;
    if (p->cmax < 0) return EDP_ERR_INVALID_ARG;
    switch (p->cost_mode) {
    case EDP_COST_PAIR:
        if (s->R > 2) return EDP_ERR_INVALID_ARG;
        break;
    case EDP_COST_PAIR_STEREO3:
        if (s->R != 3 || !I2) return EDP_ERR_INVALID_ARG;
        break;
    case EDP_COST_COMPOSITE:
        if (s->R > 2 || !I2) return EDP_ERR_INVALID_ARG;
        break;
    default:
        return EDP_ERR_INVALID_ARG;
    }
    if (p->l2 == 2 && p->cmax > (1 << 24)) return EDP_ERR_RANGE;
    return EDP_OK;
}

int run_cost(const uint8_t *I0, const uint8_t *I1, const uint8_t *I2, int W, int H, int pitch,
             const edp_label_space *s, const edp_params *p, int Q, int32_t *C, cudaStream_t st) {
    CostArgs a;
    memset(&a, 0, sizeof a);
    a.I0 = I0;
    a.I1 = I1;
    a.I2 = I2;
    a.W = W;
    a.H = H;
    a.pitch = pitch;
    a.R = s->R;
    a.Q = Q;
    a.Q0 = s->Q[0];
    a.Q1 = s->Q[1];
    a.Q2 = s->Q[2];
    for (int r = 0; r < 3; ++r) {
        a.vmin[r] = s->vmin[r];
        a.step[r] = r < s->R ? s->step[r] : 1;
    }
    a.l2 = p->l2;
    a.cmax = p->cmax;
    a.mode = p->cost_mode;
    a.C = C;
    return launch_cost(a, st) ? EDP_ERR_CUDA : EDP_OK;
}

int run_energy(const int32_t *C, const int32_t *labels, int W, int H, const edp_label_space *s,
               const edp_params *p, int Q, int64_t *out4, cudaStream_t st, const uint8_t *wh = nullptr,
               const uint8_t *wv = nullptr, const FusedImages *fi = nullptr) {
    EnergyArgs a;
    memset(&a, 0, sizeof a);
    if (fi) {  // the data term from the images (C not read)
        a.I0 = fi->I0;
        a.I1 = fi->I1;
        a.pitch = fi->pitch;
        a.v0 = fi->v0;
        a.v1 = fi->v1;
        a.t0 = fi->t0;
        a.t1 = fi->t1;
        a.cmax = fi->cmax;
        a.l2 = fi->l2;
        C = nullptr;
    }
    a.wh = wh;
    a.wv = wv;
    a.C = C;
    a.labels = labels;
    a.W = W;
    a.H = H;
    a.Q = Q;
    a.R = s->R;
    a.Q0 = s->Q[0];
    a.Q1 = s->Q[1];
    a.lam = p->lambda;
    a.g = p->g;
    a.l1 = p->l1;
    a.mode = p->prior_mode;
    a.out4 = reinterpret_cast<long long *>(out4);
    return launch_energy(a, st) ? EDP_ERR_CUDA : EDP_OK;
}

}  // namespace

extern "C" {

int edp_version(void) { return 10000; }

const char *edp_status_string(int status) {
    switch (status) {
    case EDP_OK: return "EDP_OK";
    case EDP_ERR_INVALID_ARG: return "EDP_ERR_INVALID_ARG";
    case EDP_ERR_UNSUPPORTED: return "EDP_ERR_UNSUPPORTED";
    case EDP_ERR_WORKSPACE: return "EDP_ERR_WORKSPACE";
    case EDP_ERR_RANGE: return "EDP_ERR_RANGE";
    case EDP_ERR_TIMEOUT: return "EDP_ERR_TIMEOUT";
    case EDP_ERR_CUDA: return "EDP_ERR_CUDA";
    default: return "EDP_ERR_UNKNOWN";
    }
}

int edp_set_tuning(int rows_per_block, int labels_per_lane, int warps_per_row, int general_kernel) {
    if (rows_per_block < 0 || labels_per_lane < 0 || labels_per_lane > kEM) return EDP_ERR_INVALID_ARG;
    if (warps_per_row < 0 || warps_per_row > 12) return EDP_ERR_INVALID_ARG;
    if (general_kernel < 0 || general_kernel > 5) return EDP_ERR_INVALID_ARG;
    g_tune_rb = rows_per_block;
    g_tune_e = labels_per_lane;
    g_tune_t = warps_per_row;
    g_force_general = general_kernel == 1 || general_kernel == 2;
    g_generic_team = general_kernel == 2;
    g_line_mode = general_kernel == 3 ? 1 : (general_kernel >= 4 ? 2 : 0);
    g_line_split = general_kernel == 5 ? 0 : 1;
    return EDP_OK;
}

int edp_set_fused_cost(int on) {
    if (on != 0 && on != 1) return EDP_ERR_INVALID_ARG;
    g_fused_cost = on;
    return EDP_OK;
}

int edp_set_pass_pairs(int mode) {
    if (mode < 0 || mode > 2) return EDP_ERR_INVALID_ARG;
    g_pass_pairs = mode;
    return EDP_OK;
}

int edp_last_pass_launches(void) { return g_last_launches; }

const char *edp_last_pass_kernel(void) { return g_last_kernel; }

int edp_set_batch_split(long long min_pixels) {
    if (min_pixels < 0) return EDP_ERR_INVALID_ARG;
    g_batch_alone_pixels = min_pixels > INT_MAX ? INT_MAX : (int)min_pixels;
    return EDP_OK;
}

int edp_set_spin_limit(long long polls) {
    if (polls < 0) return EDP_ERR_INVALID_ARG;
    g_spin_limit = polls ? polls : kSpinDefault;
    return EDP_OK;
}

int edp_test_hold_band(int band) {
    if (band < 0) return EDP_ERR_INVALID_ARG;
    g_hold_band = band;
    return EDP_OK;
}

int edp_set_profile_events(void *const *events, int n_events) {
    if (n_events < 0 || (n_events > 0 && !events)) return EDP_ERR_INVALID_ARG;
    g_prof_events = n_events ? events : nullptr;
    g_prof_n = n_events;
    return EDP_OK;
}

int edp_set_trace(void *device_buffer, size_t bytes) {
    if (bytes > 0 && !device_buffer) return EDP_ERR_INVALID_ARG;
    g_trace = bytes ? static_cast<unsigned long long *>(device_buffer) : nullptr;
    g_trace_bytes = bytes;
    return EDP_OK;
}

namespace {
// Coarse level of the proposal (two-axis motion spaces): the images halved
// (2x2 averages), the label space with halved offsets.
struct CoarseGeometry {
    int Wc, Hc;
    edp_label_space sc;
};
int coarse_geometry(int W, int H, const edp_label_space *s, CoarseGeometry *c) {
    if (!s || s->R != 2 || s->step[0] != 1 || s->step[1] != 1 || s->Q[2] != 1) return EDP_ERR_UNSUPPORTED;
    c->Wc = (W + 1) / 2;
    c->Hc = (H + 1) / 2;
    memset(&c->sc, 0, sizeof c->sc);
    c->sc.R = 2;
    for (int r = 0; r < 2; ++r) {
        const int lo = s->vmin[r], hi = s->vmin[r] + s->Q[r] - 1;
        const int clo = lo >= 0 ? (lo + 1) / 2 : -((-lo) / 2);  // ceil(lo / 2)
        const int chi = hi >= 0 ? hi / 2 : -((-hi + 1) / 2);     // floor(hi / 2)
        c->sc.vmin[r] = clo;
        c->sc.Q[r] = std::max(1, chi - clo + 1);
        c->sc.step[r] = 1;
    }
    c->sc.Q[2] = 1;
    c->sc.step[2] = 1;
    return EDP_OK;
}
struct CoarseLayout {
    size_t img[2], labels, solve, end;
};
CoarseLayout coarse_layout(const CoarseGeometry &c, int iters) {
    CoarseLayout L;
    L.img[0] = kHeader;
    L.img[1] = align_up(L.img[0] + (size_t)c.Wc * c.Hc);
    L.labels = align_up(L.img[1] + (size_t)c.Wc * c.Hc);
    L.solve = align_up(L.labels + (size_t)c.Wc * c.Hc * 4);
    L.end = L.solve + images_layout(c.Wc, c.Hc, c.sc.Q[0] * c.sc.Q[1], 2, iters).end;
    return L;
}
}  // namespace

size_t edp_workspace_size(int op, int W, int H, const edp_label_space *space, const edp_params *params) {
    Geometry g;
    if (W < 1 || H < 1 || check_space(space, &g) || !params) return 0;
    const int iters = std::max(1, params->iters);
    switch (op) {
    case EDP_OP_SCANLINE_DP:
        return align_up(kHeader + (size_t)W * H * g.Q * ptr_bytes_for(g.Q));
    case EDP_OP_SOLVE:
        return solve_layout(W, H, g.Q, g.R, iters).end;
    case EDP_OP_SOLVE_IMAGES:
        return images_layout(W, H, g.Q, g.R, iters).end;
    case EDP_OP_SCANLINE_MARGINALS:
        return align_up(kHeader + (size_t)W * H * g.Q * 4) + align_up((size_t)W * H * g.Q * 4);
    case EDP_OP_COARSE: {
        CoarseGeometry c;
        if (coarse_geometry(W, H, space, &c)) return 0;
        return coarse_layout(c, iters).end;
    }
    default:
        return 0;
    }
}

int edp_cost_volume(const uint8_t *I0, const uint8_t *I1, const uint8_t *I2, int W, int H, int pitch,
                    const edp_label_space *space, const edp_params *params, int32_t *C, edp_stream_t stream) {
    Geometry g;
    int rc = check_space(space, &g);
    if (rc) return rc;
    if ((rc = check_images(I0, I1, I2, W, H, pitch, space, params))) return rc;
    if (!C) return EDP_ERR_INVALID_ARG;
    return run_cost(I0, I1, I2, W, H, pitch, space, params, g.Q, C, (cudaStream_t)stream);
}

int edp_scanline_dp(const int32_t *C, int W, int H, const edp_label_space *space, const edp_params *params,
                    int32_t *labels, int64_t *row_energy, void *ws, size_t ws_bytes, edp_stream_t stream) {
    Geometry g;
    int rc = check_space(space, &g);
    if (rc) return rc;
    if ((rc = check_prior(params))) return rc;
    if (!C || !labels || !ws || W < 1 || H < 1) return EDP_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return EDP_ERR_INVALID_ARG;
    if (params->l1 != 1 && g.R != 1) return EDP_ERR_UNSUPPORTED;  // quadratic taps: one label axis
    if (ws_bytes < edp_workspace_size(EDP_OP_SCANLINE_DP, W, H, space, params)) return EDP_ERR_WORKSPACE;
    // S values along a row stay below W * (cmax + R * lambda * g)
    if ((long long)W * (params->cmax + (long long)g.R * cap_value(params)) >= (1LL << 29)) return EDP_ERR_RANGE;
    if (params->lambda > (1 << 20)) return EDP_ERR_RANGE;
    const int pb = ptr_bytes_for(g.Q);
    DpConfig cfg;
    bool psm = false;
    if ((rc = configure(g, H, true, W, pb, &psm, &cfg))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = cuda_status(cudaMemsetAsync(ws, 0, kHeader, st)))) return rc;
    ScanArgs a;
    memset(&a, 0, sizeof a);
    a.C = C;
    a.labels = labels;
    a.row_energy = reinterpret_cast<long long *>(row_energy);
    a.ptr = static_cast<unsigned char *>(ws) + kHeader;
    a.ptr_bytes = pb;
    a.ptr_in_smem = psm;
    a.W = W;
    a.H = H;
    a.Q = g.Q;
    a.R = g.R;
    for (int r = 0; r < 3; ++r) a.ax[r] = cfg.ax[r];
    a.lam = params->lambda;
    a.capv = (int)cap_value(params);
    a.mode = params->prior_mode;
    a.l1 = params->l1;
    a.g = params->g;
    a.RB = cfg.RB;
    const int grid = (H + cfg.RB - 1) / cfg.RB;
    return launch_scanline(a, cfg.em, cfg.threads, cfg.smem, grid, st) ? EDP_ERR_CUDA : EDP_OK;
}

int edp_scanline_marginals(const int32_t *C, int W, int H, const edp_label_space *space, const edp_params *params,
                           int32_t *labels, int32_t *marginals, void *ws, size_t ws_bytes, edp_stream_t stream) {
    Geometry g;
    int rc = check_space(space, &g);
    if (rc) return rc;
    if ((rc = check_prior(params))) return rc;
    if (!C || !labels || !ws || W < 1 || H < 1) return EDP_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return EDP_ERR_INVALID_ARG;
    if (params->l1 != 1 && g.R != 1) return EDP_ERR_UNSUPPORTED;  // quadratic taps: one label axis
    if (ws_bytes < edp_workspace_size(EDP_OP_SCANLINE_MARGINALS, W, H, space, params)) return EDP_ERR_WORKSPACE;
    // forward and backward sums stay below W * (cmax + R * lambda * g): their
    // sum minus the cost fits int32
    if ((long long)W * (params->cmax + (long long)g.R * cap_value(params)) >= (1LL << 29)) return EDP_ERR_RANGE;
    if (params->lambda > (1 << 20)) return EDP_ERR_RANGE;
    DpConfig cfg;
    bool psm = false;
    if ((rc = configure(g, H, true, W, 0, &psm, &cfg))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *w = static_cast<unsigned char *>(ws);
    int *F = reinterpret_cast<int *>(w + kHeader);
    int *B = reinterpret_cast<int *>(w + align_up(kHeader + (size_t)W * H * g.Q * 4));
    ScanArgs a;
    memset(&a, 0, sizeof a);
    a.C = C;
    a.labels = labels;
    a.W = W;
    a.H = H;
    a.Q = g.Q;
    a.R = g.R;
    for (int r = 0; r < 3; ++r) a.ax[r] = cfg.ax[r];
    a.lam = params->lambda;
    a.capv = (int)cap_value(params);
    a.mode = params->prior_mode;
    a.l1 = params->l1;
    a.g = params->g;
    a.RB = cfg.RB;
    a.no_ptr = 1;
    const int grid = (H + cfg.RB - 1) / cfg.RB;
    a.sums = F;
    a.reverse = 0;
    if (launch_scanline(a, cfg.em, cfg.threads, cfg.smem, grid, st)) return EDP_ERR_CUDA;
    a.sums = B;
    a.reverse = 1;
    if (launch_scanline(a, cfg.em, cfg.threads, cfg.smem, grid, st)) return EDP_ERR_CUDA;
    return launch_marginal_argmin(C, F, B, (long long)W * H, g.Q, labels, marginals, st) ? EDP_ERR_CUDA : EDP_OK;
}

int edp_solve(const int32_t *C, int W, int H, const edp_label_space *space, const edp_params *params,
              int32_t *labels, void *ws, size_t ws_bytes, edp_stream_t stream) {
    Geometry g;
    int rc = check_space(space, &g);
    if (rc) return rc;
    if ((rc = check_prior(params))) return rc;
    if (!C || !labels || !ws || W < 1 || H < 1 || params->iters < 1) return EDP_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return EDP_ERR_INVALID_ARG;
    // l1 = 2 (quadratic taps) is planned per kernel form; unsupported forms return EDP_ERR_UNSUPPORTED
    if (ws_bytes < edp_workspace_size(EDP_OP_SOLVE, W, H, space, params)) return EDP_ERR_WORKSPACE;
    if ((rc = check_range(W, H, g, params))) return rc;
    return run_solve(C, W, H, g, params, labels, static_cast<unsigned char *>(ws), (cudaStream_t)stream);
}

int edp_edge_weights(const uint8_t *I, int W, int H, int pitch, int threshold, int factor, uint8_t *wh, uint8_t *wv,
                     edp_stream_t stream) {
    if (!I || !wh || !wv || W < 1 || H < 1 || pitch < W) return EDP_ERR_INVALID_ARG;
    if (factor < 0 || factor > 255 || threshold < 0) return EDP_ERR_INVALID_ARG;
    return launch_edge_weights(I, W, H, pitch, threshold, factor, wh, wv, (cudaStream_t)stream) ? EDP_ERR_CUDA
                                                                                                 : EDP_OK;
}

int edp_solve_weighted(const int32_t *C, int W, int H, const edp_label_space *space, const edp_params *params,
                       const uint8_t *wh, const uint8_t *wv, int max_weight, int32_t *labels, void *ws,
                       size_t ws_bytes, edp_stream_t stream) {
    Geometry g;
    int rc = check_space(space, &g);
    if (rc) return rc;
    if ((rc = check_prior(params))) return rc;
    if (!C || !wh || !wv || !labels || !ws || W < 1 || H < 1 || params->iters < 1) return EDP_ERR_INVALID_ARG;
    if (max_weight < 0 || max_weight > 255) return EDP_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return EDP_ERR_INVALID_ARG;
    if (ws_bytes < edp_workspace_size(EDP_OP_SOLVE, W, H, space, params)) return EDP_ERR_WORKSPACE;
    if ((rc = check_range(W, H, g, params))) return rc;
    // the int32 range bound of the heaviest edge: lambda times the largest multiplier
    edp_params pw = *params;
    pw.lambda = params->lambda * std::max(1, max_weight);
    if ((rc = check_range(W, H, g, &pw))) return rc;
    return run_solve(C, W, H, g, params, labels, static_cast<unsigned char *>(ws), (cudaStream_t)stream, wh, wv);
}

int edp_energy_weighted(const int32_t *C, const int32_t *labels, int W, int H, const edp_label_space *space,
                        const edp_params *params, const uint8_t *wh, const uint8_t *wv, int64_t *out4,
                        edp_stream_t stream) {
    Geometry g;
    int rc = check_space(space, &g);
    if (rc) return rc;
    if ((rc = check_prior(params))) return rc;
    if (!labels || !out4 || !wh || !wv || W < 1 || H < 1) return EDP_ERR_INVALID_ARG;
    return run_energy(C, labels, W, H, space, params, g.Q, out4, (cudaStream_t)stream, wh, wv);
}

int edp_energy(const int32_t *C, const int32_t *labels, int W, int H, const edp_label_space *space,
               const edp_params *params, int64_t *out4, edp_stream_t stream) {
    Geometry g;
    int rc = check_space(space, &g);
    if (rc) return rc;
    if ((rc = check_prior(params))) return rc;
    if (!labels || !out4 || W < 1 || H < 1) return EDP_ERR_INVALID_ARG;
    return run_energy(C, labels, W, H, space, params, g.Q, out4, (cudaStream_t)stream);
}

int edp_solve_images(const uint8_t *I0, const uint8_t *I1, const uint8_t *I2, int W, int H, int pitch,
                     const edp_label_space *space, const edp_params *params, int32_t *labels, int64_t *energy4,
                     void *ws, size_t ws_bytes, edp_stream_t stream) {
    Geometry g;
    int rc = check_space(space, &g);
    if (rc) return rc;
    if ((rc = check_prior(params))) return rc;
    if ((rc = check_images(I0, I1, I2, W, H, pitch, space, params))) return rc;
    if (!labels || !ws || params->iters < 1) return EDP_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return EDP_ERR_INVALID_ARG;
    // l1 = 2 (quadratic taps) is planned per kernel form; unsupported forms return EDP_ERR_UNSUPPORTED
    if (ws_bytes < edp_workspace_size(EDP_OP_SOLVE_IMAGES, W, H, space, params)) return EDP_ERR_WORKSPACE;
    if ((rc = check_range(W, H, g, params))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *w = static_cast<unsigned char *>(ws);
    const ImagesLayout L = images_layout(W, H, g.Q, g.R, params->iters);
    int32_t *C = reinterpret_cast<int32_t *>(w + L.C);
    // the pair cost of a two-axis space on the split line kernel: computed
    // from the images inside the scan passes and the energy, no cost volume
    bool fuse = false;
    if (g_fused_cost && params->cost_mode == 0 && space->R == 2) {
        SolvePlan P;
        fuse = plan_solve(C, W, H, g, params, labels, w, &P) == EDP_OK && P.line && P.split;
    }
    const FusedImages fi = fused_images(I0, I1, pitch, space, params);
    if (!fuse && (rc = run_cost(I0, I1, I2, W, H, pitch, space, params, g.Q, C, st))) return rc;
    if ((rc = run_solve(C, W, H, g, params, labels, w, st, nullptr, nullptr, fuse ? &fi : nullptr))) return rc;
    if (energy4) rc = run_energy(C, labels, W, H, space, params, g.Q, energy4, st, nullptr, nullptr, fuse ? &fi : nullptr);
    return rc;
}

int edp_solve_images_host(const uint8_t *I0_host, const uint8_t *I1_host, const uint8_t *I2_host, int W,
                          int H, const edp_label_space *space, const edp_params *params, int32_t *labels_host,
                          int64_t *energy4_host, void *ws, size_t ws_bytes, edp_stream_t stream) {
    Geometry g;
    int rc = check_space(space, &g);
    if (rc) return rc;
    if (!I0_host || !I1_host || !labels_host || !ws || W < 1 || H < 1 || !params) return EDP_ERR_INVALID_ARG;
    if (ws_bytes < edp_workspace_size(EDP_OP_SOLVE_IMAGES, W, H, space, params)) return EDP_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *w = static_cast<unsigned char *>(ws);
    const ImagesLayout L = images_layout(W, H, g.Q, g.R, std::max(1, params->iters));
    const size_t npix = (size_t)W * H;
    const uint8_t *hin[3] = {I0_host, I1_host, I2_host};
    for (int k = 0; k < 3; ++k)
        if (hin[k] && (rc = cuda_status(cudaMemcpyAsync(w + L.img[k], hin[k], npix, cudaMemcpyHostToDevice, st))))
            return rc;
    int32_t *labels = reinterpret_cast<int32_t *>(w + L.labels);
    int64_t *energy = reinterpret_cast<int64_t *>(w + L.energy);
    rc = edp_solve_images(w + L.img[0], w + L.img[1], I2_host ? w + L.img[2] : nullptr, W, H, W, space, params,
                          labels, energy, ws, ws_bytes, stream);
    if (rc) return rc;
    if ((rc = cuda_status(cudaMemcpyAsync(labels_host, labels, npix * 4, cudaMemcpyDeviceToHost, st)))) return rc;
    if (energy4_host &&
        (rc = cuda_status(cudaMemcpyAsync(energy4_host, energy, 4 * 8, cudaMemcpyDeviceToHost, st))))
        return rc;
    return cuda_status(cudaStreamSynchronize(st));
}

namespace {
// batch workspace: control block (status | queue | done[kMaxBatch][4*iters])
// followed by each resident problem's solve workspace and cost volume
size_t batch_ctrl_bytes(int iters) { return align_up(kHeader + 256 + (size_t)kMaxBatch * 4 * iters * 4); }

size_t problem_bytes(const edp_problem &pr, const Geometry &g) {
    const int iters = std::max(1, pr.params.iters);
    return align_up(solve_layout(pr.W, pr.H, g.Q, g.R, iters).end + (size_t)pr.W * pr.H * g.Q * 4);
}

int check_problem(const edp_problem &pr, Geometry *g) {
    int rc = check_space(&pr.space, g);
    if (rc) return rc;
    if ((rc = check_prior(&pr.params))) return rc;
    if ((rc = check_images(pr.I0, pr.I1, pr.I2, pr.W, pr.H, pr.pitch, &pr.space, &pr.params))) return rc;
    if (!pr.labels || pr.params.iters < 1) return EDP_ERR_INVALID_ARG;
    // l1 = 2 (quadratic taps) is planned per kernel form; unsupported forms return EDP_ERR_UNSUPPORTED
    return check_range(pr.W, pr.H, *g, &pr.params);
}

// One persistent launch over the problems idx[0..n) of a chunk; problem
// idx[k] has its region (solve workspace, then cost volume) at ws + offs[k].
int run_wave(const edp_problem *probs_all, const Geometry *geo_all, const int *idx, const size_t *offs, int n,
             int iters, unsigned char *ws, cudaStream_t st) {
    const size_t ctrl = batch_ctrl_bytes(iters);
    int *status = reinterpret_cast<int *>(ws);
    ZeroBatch zb;
    memset(&zb, 0, sizeof zb);
    zb.ptr[zb.n] = ws;
    zb.bytes[zb.n++] = ctrl;
    CostBatch cb;
    memset(&cb, 0, sizeof cb);
    EnergyBatch eb;
    memset(&eb, 0, sizeof eb);
    static BatchArgs B;  // too large for the stack of some callers; filled and copied into the launch
    memset(&B, 0, sizeof B);
    B.n = n;
    // the wave's bands share the blocks, so a paired band holding its block twice
    // as long costs more than the shorter wavefront saves (measured on the
    // 64-problem batch): pairs only when asked for explicitly
    B.pairs = g_pass_pairs == 1;
    B.slots = (B.pairs ? 2 : 4) * iters;
    B.queue = reinterpret_cast<unsigned *>(ws + kHeader);
    B.done = reinterpret_cast<unsigned *>(ws + kHeader + 256);
    B.status = status;
    B.spin_limit = g_spin_limit;
    long long max_entries = 0, max_pixels = 0;
    // one block shape for the wave: 8 warps (one-axis bands of 8 rows, or
    // teams of the multi-axis body)
    const int threads = 256;
    int quad = 0, gen = 0;
    size_t smem = 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    static SolvePlan plans[kMaxBatch];
    for (int k = 0; k < n; ++k) {
        const edp_problem &pr = probs_all[idx[k]];
        const Geometry &g = geo_all[idx[k]];
        unsigned char *pws = ws + offs[k];
        const SolveLayout L = solve_layout(pr.W, pr.H, g.Q, g.R, iters);
        int32_t *C = reinterpret_cast<int32_t *>(pws + L.end);
        int rc = plan_solve(C, pr.W, pr.H, g, &pr.params, pr.labels, pws, &plans[k], threads);
        if (rc) return rc;
        if (plans[k].r1 ? plans[k].o.l1 == 2 : plans[k].ta.l1 == 2) quad = 1;
        if (!plans[k].r1 && !plans[k].ta.lean) gen = 1;
        smem = std::max(smem, plans[k].smem);
    }
    const int lm = quad ? 2 : 33;  // batched build: quadratic-prior bodies only when needed
    const int occ = std::max(1, edp_batched_occupancy(lm, gen, threads, smem));
    // work items run problem by problem inside each pass: the largest problems
    // (longest wavefronts) first, so that small ones fill in behind them
    int order[kMaxBatch], slot_of[kMaxBatch];
    for (int k = 0; k < n; ++k) order[k] = k;
    auto work = [&](int k) {
        const edp_problem &pr = probs_all[idx[k]];
        return (double)pr.W * pr.H * geo_all[idx[k]].Q;
    };
    std::stable_sort(order, order + n, [&](int a, int b) { return work(a) > work(b); });
    for (int j = 0; j < n; ++j) slot_of[order[j]] = j;
    for (int j = 0; j < n; ++j) B.prefix[j + 1] = B.prefix[j] + plans[order[j]].nbands;
    for (int k = 0; k < n; ++k) {
        const edp_problem &pr = probs_all[idx[k]];
        const Geometry &g = geo_all[idx[k]];
        unsigned char *pws = ws + offs[k];
        const SolveLayout L = solve_layout(pr.W, pr.H, g.Q, g.R, iters);
        int32_t *C = reinterpret_cast<int32_t *>(pws + L.end);
        const SolvePlan &P = plans[k];
        if (!P.r1 && team_ring(B.pairs ? 2 * pr.W : pr.W, occ * sms) > P.ta.ring) return EDP_ERR_UNSUPPORTED;
        BatchProblem &bp = B.p[slot_of[k]];
        bp.r1 = P.r1;
        bp.nbands = P.nbands;
        bp.iters = iters;
        bp.laps = P.laps;
        bp.cons = reinterpret_cast<unsigned *>(pws + L.cons);
        if (P.r1) {
            bp.o = P.o;
            bp.o.status = status;
        } else {
            bp.t = P.ta;
            bp.t.status = status;
        }
        zb.ptr[zb.n] = pws;
        zb.bytes[zb.n++] = control_bytes(P, pr.W, g.Q);
        CostArgs &c = cb.c[k];
        c.I0 = pr.I0;
        c.I1 = pr.I1;
        c.I2 = pr.I2;
        c.W = pr.W;
        c.H = pr.H;
        c.pitch = pr.pitch;
        c.R = pr.space.R;
        c.Q = g.Q;
        c.Q0 = pr.space.Q[0];
        c.Q1 = pr.space.Q[1];
        c.Q2 = pr.space.Q[2];
        for (int r = 0; r < 3; ++r) {
            c.vmin[r] = pr.space.vmin[r];
            c.step[r] = r < pr.space.R ? pr.space.step[r] : 1;
        }
        c.l2 = pr.params.l2;
        c.cmax = pr.params.cmax;
        c.mode = pr.params.cost_mode;
        c.C = C;
        EnergyArgs &e = eb.e[k];
        e.C = C;
        e.labels = pr.labels;
        e.W = pr.W;
        e.H = pr.H;
        e.Q = g.Q;
        e.R = pr.space.R;
        e.Q0 = pr.space.Q[0];
        e.Q1 = pr.space.Q[1];
        e.lam = pr.params.lambda;
        e.g = pr.params.g;
        e.l1 = pr.params.l1;
        e.mode = pr.params.prior_mode;
        e.out4 = reinterpret_cast<long long *>(pr.energy4);
        if (pr.energy4) {
            zb.ptr[zb.n] = pr.energy4;
            zb.bytes[zb.n++] = 4 * sizeof(int64_t);
        }
        max_entries = std::max(max_entries, (long long)pr.W * pr.H * g.Q);
        max_pixels = std::max(max_pixels, (long long)pr.W * pr.H);
    }
    B.per_slot = B.prefix[n];
    cb.n = n;
    eb.n = n;
    if (launch_zero_batched(zb, st)) return EDP_ERR_CUDA;
    if (launch_cost_batched(cb, max_entries, st)) return EDP_ERR_CUDA;
    const int grid = std::max(1, std::min(B.slots * B.per_slot, occ * sms));
    if (launch_edp_batched(B, lm, gen, threads, smem, grid, st)) return EDP_ERR_CUDA;
    if (launch_energy_batched(eb, max_pixels, st)) return EDP_ERR_CUDA;
    return EDP_OK;
}
}  // namespace

size_t edp_batch_workspace_size(const edp_problem *probs, int n) {
    if (!probs || n < 1) return 0;
    size_t total = 0;
    int iters = 1;
    for (int k = 0; k < n; ++k) {
        Geometry g;
        if (check_space(&probs[k].space, &g) || probs[k].W < 1 || probs[k].H < 1) return 0;
        total += problem_bytes(probs[k], g);
        iters = std::max(iters, probs[k].params.iters);
    }
    return batch_ctrl_bytes(iters) + total;
}

int edp_solve_batched(const edp_problem *probs, int n, void *ws, size_t ws_bytes, edp_stream_t stream) {
    if (!probs || n < 1 || !ws) return EDP_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return EDP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *w = static_cast<unsigned char *>(ws);
    Geometry geo_small[64];
    Geometry *geo = geo_small;
    if (n > 64) return EDP_ERR_UNSUPPORTED;  // larger batches: call again per 64 problems
    for (int k = 0; k < n; ++k) {
        int rc = check_problem(probs[k], &geo[k]);
        if (rc) return rc;
    }
    int first = 0;
    while (first < n) {
        const int iters = probs[first].params.iters;
        const size_t ctrl = batch_ctrl_bytes(iters);
        size_t used = ctrl;
        int cnt = 0;
        while (first + cnt < n && cnt < kMaxBatch && probs[first + cnt].params.iters == iters) {
            const size_t b = problem_bytes(probs[first + cnt], geo[first + cnt]);
            if (used + b > ws_bytes) break;
            used += b;
            ++cnt;
        }
        if (cnt == 0) return EDP_ERR_WORKSPACE;
        // regions of the chunk's problems; problems that fill the GPU on their
        // own run with their own launch shapes (one after another), the others
        // share one persistent launch
        int widx[kMaxBatch];
        size_t woff[kMaxBatch];
        int nw = 0;
        size_t off = ctrl;
        for (int k = first; k < first + cnt; ++k) {
            const edp_problem &pr = probs[k];
            const Geometry &g = geo[k];
            if (g_batch_alone_pixels > 0 && (long long)pr.W * pr.H >= g_batch_alone_pixels) {
                unsigned char *pws = w + off;
                int32_t *C = reinterpret_cast<int32_t *>(pws + solve_layout(pr.W, pr.H, g.Q, g.R, iters).end);
                int rc = run_cost(pr.I0, pr.I1, pr.I2, pr.W, pr.H, pr.pitch, &pr.space, &pr.params, g.Q, C, st);
                if (!rc) rc = run_solve(C, pr.W, pr.H, g, &pr.params, pr.labels, pws, st);
                if (!rc && pr.energy4) rc = run_energy(C, pr.labels, pr.W, pr.H, &pr.space, &pr.params, g.Q, pr.energy4, st);
                if (rc) return rc;
            } else {
                widx[nw] = k;
                woff[nw++] = off;
            }
            off += problem_bytes(pr, g);
        }
        if (nw > 0) {
            int rc = run_wave(probs, geo, widx, woff, nw, iters, w, st);
            if (rc) return rc;
        }
        first += cnt;
    }
    return EDP_OK;
}

namespace {
int check_window(const edp_label_space *space, const edp_params *params, int win, Geometry *g) {
    int rc = check_space(space, g);
    if (rc) return rc;
    if ((rc = check_prior(params))) return rc;
    if (space->R > 2) return EDP_ERR_UNSUPPORTED;
    if (win < 1 || (win & 1) == 0 || win > 15) return EDP_ERR_UNSUPPORTED;
    for (int r = 0; r < space->R; ++r)
        if (space->Q[r] < win) return EDP_ERR_INVALID_ARG;
    return EDP_OK;
}
}  // namespace

size_t edp_workspace_size_windowed(int W, int H, const edp_label_space *space, const edp_params *params,
                                   int win) {
    Geometry g;
    if (W < 1 || H < 1 || check_window(space, params, win, &g)) return 0;
    const int Qw = space->R == 2 ? win * win : win;
    return solve_layout(W, H, Qw, space->R, std::max(1, params->iters)).end;
}

int edp_cost_window(const uint8_t *I0, const uint8_t *I1, const uint8_t *I2, int W, int H, int pitch,
                    const edp_label_space *space, const edp_params *params, const int32_t *centre, int win,
                    int32_t *Cw, edp_stream_t stream) {
    Geometry g;
    int rc = check_window(space, params, win, &g);
    if (rc) return rc;
    if ((rc = check_images(I0, I1, I2, W, H, pitch, space, params))) return rc;
    if (params->cost_mode == EDP_COST_PAIR_STEREO3) return EDP_ERR_UNSUPPORTED;
    if (!centre || !Cw) return EDP_ERR_INVALID_ARG;
    CostArgs a;
    memset(&a, 0, sizeof a);
    a.I0 = I0;
    a.I1 = I1;
    a.I2 = I2;
    a.W = W;
    a.H = H;
    a.pitch = pitch;
    a.R = space->R;
    a.Q0 = space->Q[0];
    a.Q1 = space->Q[1];
    for (int r = 0; r < 3; ++r) {
        a.vmin[r] = space->vmin[r];
        a.step[r] = r < space->R ? space->step[r] : 1;
    }
    a.l2 = params->l2;
    a.cmax = params->cmax;
    a.mode = params->cost_mode;
    a.C = Cw;
    return launch_cost_window(a, centre, win, (cudaStream_t)stream) ? EDP_ERR_CUDA : EDP_OK;
}

int edp_solve_windowed(const int32_t *Cw, const int32_t *centre, int win, int W, int H,
                       const edp_label_space *space, const edp_params *params, int32_t *labels, void *ws,
                       size_t ws_bytes, edp_stream_t stream) {
    Geometry g;
    int rc = check_window(space, params, win, &g);
    if (rc) return rc;
    if (!Cw || !centre || !labels || !ws || W < 1 || H < 1 || params->iters < 1) return EDP_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return EDP_ERR_INVALID_ARG;
    if (ws_bytes < edp_workspace_size_windowed(W, H, space, params, win)) return EDP_ERR_WORKSPACE;
    Geometry gw = g;
    gw.R = space->R;
    if ((rc = check_range(W, H, gw, params))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *w = static_cast<unsigned char *>(ws);
    const int Qw = space->R == 2 ? win * win : win;
    // the multi-axis pass kernel in its windowed form: one warp per row, the
    // workspace laid out as edp_solve's with Q = Qw
    const SolveLayout L = solve_layout(W, H, Qw, space->R, params->iters);
    TeamArgs a;
    memset(&a, 0, sizeof a);
    a.C = Cw;
    for (int k = 0; k < 4; ++k) a.M[k] = reinterpret_cast<int *>(w + L.msg[k]);
    a.labels = labels;
    a.ll = reinterpret_cast<int2 *>(w + L.ll);
    a.status = reinterpret_cast<int *>(w);
    a.W = W;
    a.H = H;
    a.Q = Qw;
    a.Qm = L.Qm;
    a.R = space->R;
    a.lam = params->lambda;
    a.capv = (int)cap_value(params);
    a.mode = params->prior_mode;
    a.T = 1;
    int NT = g_tune_rb > 0 ? g_tune_rb : 8;
    NT = std::max(1, std::min(NT, std::min(8, H)));  // the windowed builds take <= 256 threads
    a.nbuf = 3;
    a.kmb = 4;
    // (the windowed form always has the two transpose buffers: R = 2 in the size)
    while (NT > 1 && pass_team_smem(NT, L.Qm, 2, a.nbuf, a.kmb) > (size_t)kMaxSmem) --NT;
    const size_t smem = pass_team_smem(NT, L.Qm, 2, a.nbuf, a.kmb);
    if (smem > (size_t)kMaxSmem) return EDP_ERR_UNSUPPORTED;
    a.NT = NT;
    a.ring = team_ring(2 * W, kResidentMin);
    a.win = win;
    a.l1 = params->l1;
    a.g = params->g;
    a.centre = centre;
    a.Q0w = space->Q[0];
    a.Q1w = space->Q[1];
    a.em = params->l1;  // the windowed build of this prior power
    a.nbands = (H + NT - 1) / NT;
    a.spin_limit = g_spin_limit;
    const int laps = (W + a.ring - 1) / a.ring;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int occ = std::max(1, edp_pass_team_occupancy(a.em, 0, 1, 32 * NT, smem));
    a.grid = std::min(a.nbands, occ * sms);
    if (a.grid < a.nbands && team_ring(2 * W, a.grid) > a.ring) return EDP_ERR_UNSUPPORTED;
    if ((rc = cuda_status(cudaMemsetAsync(w, 0, L.ll + (size_t)a.nbands * a.ring * L.Qm * 8, st)))) return rc;
    const bool pairs = pairs_for(a.grid >= a.nbands);
    const int per_it = pairs ? 2 : 4;
    g_last_launches = per_it * params->iters;
    g_last_kernel = "edp_pass_team_kernel";
    for (int it = 0; it < params->iters; ++it)
        for (int k = 0; k < per_it; ++k) {
            const int launch = it * per_it + k;
            TeamArgs b = a;
            const int slot = it * 4 + set_launch(b, it, k, params->iters, pairs);
            b.cons = reinterpret_cast<unsigned *>(w + L.cons) + (size_t)slot * H;
            b.tag0 = 1 + slot * laps;
            b.band_counter = reinterpret_cast<unsigned *>(w + L.counters) + slot;
            const bool prof = g_prof_events && 2 * launch + 1 < g_prof_n;
            if (prof && cudaEventRecord((cudaEvent_t)g_prof_events[2 * launch], st) != cudaSuccess)
                return EDP_ERR_CUDA;
            if (launch_edp_pass_team(b, 32 * NT, smem, st)) return EDP_ERR_CUDA;
            if (prof && cudaEventRecord((cudaEvent_t)g_prof_events[2 * launch + 1], st) != cudaSuccess)
                return EDP_ERR_CUDA;
        }
    return EDP_OK;
}

int edp_wta(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch, const edp_label_space *space,
            const edp_params *params, int radius, int32_t *labels, int32_t *cost, edp_stream_t stream) {
    Geometry g;
    int rc = check_space(space, &g);
    if (rc) return rc;
    if ((rc = check_images(I0, I1, nullptr, W, H, pitch, space, params))) return rc;
    if (params->cost_mode != EDP_COST_PAIR || space->R > 2) return EDP_ERR_UNSUPPORTED;
    if (!labels || radius < 0 || radius > 15) return EDP_ERR_INVALID_ARG;
    CostArgs a;
    memset(&a, 0, sizeof a);
    a.I0 = I0;
    a.I1 = I1;
    a.W = W;
    a.H = H;
    a.pitch = pitch;
    a.R = space->R;
    a.Q = g.Q;
    a.Q0 = space->Q[0];
    a.Q1 = space->Q[1];
    for (int r = 0; r < 3; ++r) {
        a.vmin[r] = space->vmin[r];
        a.step[r] = r < space->R ? space->step[r] : 1;
    }
    a.l2 = params->l2;
    a.cmax = params->cmax;
    return wta_launch(a, radius, labels, cost, (cudaStream_t)stream) ? EDP_ERR_CUDA : EDP_OK;
}

long long edp_net_param_count(void) { return net_param_count(); }

size_t edp_net_workspace_size(int N, int H, int W) {
    if (N < 1 || H < 1 || W < 1) return 0;
    return net_workspace_bytes((long long)N * H * W);
}

size_t edp_net_activation_offset(int N, int H, int W, int layer) {
    if (N < 1 || H < 1 || W < 1 || layer < 0 || layer > 5) return (size_t)-1;
    return net_activation_offset((long long)N * H * W, layer);
}

int edp_net_forward(const float *params, const void *x, int N, int H, int W, float *out, void *ws, size_t ws_bytes,
                    edp_stream_t stream) {
    if (!params || !x || !out || !ws || N < 1 || H < 1 || W < 1) return EDP_ERR_INVALID_ARG;
    if (ws_bytes < edp_net_workspace_size(N, H, W)) return EDP_ERR_WORKSPACE;
    return net_forward(params, x, N, H, W, out, static_cast<unsigned char *>(ws), (cudaStream_t)stream)
               ? EDP_ERR_CUDA
               : EDP_OK;
}

int edp_net_backward(const float *params, const float *out, const float *target, int N, int H, int W, float *grad,
                     double *loss, void *ws, size_t ws_bytes, edp_stream_t stream) {
    if (!params || !out || !target || !grad || !loss || !ws || N < 1 || H < 1 || W < 1) return EDP_ERR_INVALID_ARG;
    if (ws_bytes < edp_net_workspace_size(N, H, W)) return EDP_ERR_WORKSPACE;
    return net_backward(params, out, target, N, H, W, grad, loss, static_cast<unsigned char *>(ws),
                        (cudaStream_t)stream)
               ? EDP_ERR_CUDA
               : EDP_OK;
}

int edp_set_net_tensor_cores(int on) {
    if (on != 0 && on != 1) return EDP_ERR_INVALID_ARG;
    net_set_tensor_cores(on);
    return EDP_OK;
}

int edp_net_get_device_status(const void *ws, size_t ws_bytes, int *status, edp_stream_t stream) {
    if (!ws || !status || ws_bytes < net_status_offset() + sizeof(int)) return EDP_ERR_INVALID_ARG;
    const auto *p = static_cast<const unsigned char *>(ws) + net_status_offset();
    if (cudaMemcpyAsync(status, p, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
        return EDP_ERR_CUDA;
    return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? EDP_OK : EDP_ERR_CUDA;
}

int edp_net_adam(float *params, const float *grad, float *m, float *v, float lr, float beta1, float beta2, float eps,
                 int step, edp_stream_t stream) {
    if (!params || !grad || !m || !v || step < 1) return EDP_ERR_INVALID_ARG;
    return net_adam_step(params, grad, m, v, net_param_count(), lr, beta1, beta2, eps, step, (cudaStream_t)stream)
               ? EDP_ERR_CUDA
               : EDP_OK;
}

int edp_net_features(const uint8_t *I0, const uint8_t *I1, const int32_t *wta_labels, const int32_t *wta_cost,
                     int W, int H, const edp_label_space *space, float scale, float cmax, void *x,
                     edp_stream_t stream) {
    if (!I0 || !I1 || !wta_labels || !wta_cost || !x || !space || W < 1 || H < 1) return EDP_ERR_INVALID_ARG;
    if (space->R != 2 || !(scale > 0.f) || !(cmax > 0.f)) return EDP_ERR_INVALID_ARG;
    return net_features_launch(I0, I1, wta_labels, wta_cost, W, H, space->Q[0], space->Q[1], scale, cmax, x,
                               (cudaStream_t)stream)
               ? EDP_ERR_CUDA
               : EDP_OK;
}

int edp_net_centres(const float *out, int n, const edp_label_space *space, int32_t *centre, edp_stream_t stream) {
    if (!out || !centre || !space || n < 1 || space->R != 2) return EDP_ERR_INVALID_ARG;
    return net_centres_launch(out, n, space->Q[0], space->Q[1], centre, (cudaStream_t)stream) ? EDP_ERR_CUDA
                                                                                                : EDP_OK;
}

int edp_coarse_labels(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch, const edp_label_space *space,
                      const edp_params *params, int32_t *labels, void *ws, size_t ws_bytes, edp_stream_t stream) {
    Geometry g;
    int rc = check_space(space, &g);
    if (rc) return rc;
    if ((rc = check_prior(params))) return rc;
    if ((rc = check_images(I0, I1, nullptr, W, H, pitch, space, params))) return rc;
    if (!labels || !ws || params->iters < 1) return EDP_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return EDP_ERR_INVALID_ARG;
    CoarseGeometry c;
    if ((rc = coarse_geometry(W, H, space, &c))) return rc;
    if (ws_bytes < edp_workspace_size(EDP_OP_COARSE, W, H, space, params)) return EDP_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *w = static_cast<unsigned char *>(ws);
    const CoarseLayout L = coarse_layout(c, params->iters);
    uint8_t *h0 = w + L.img[0], *h1 = w + L.img[1];
    int32_t *lc = reinterpret_cast<int32_t *>(w + L.labels);
    if (pyr_down2_launch(I0, W, H, pitch, h0, st) || pyr_down2_launch(I1, W, H, pitch, h1, st)) return EDP_ERR_CUDA;
    rc = edp_solve_images(h0, h1, nullptr, c.Wc, c.Hc, c.Wc, &c.sc, params, lc, nullptr, w + L.solve, L.end - L.solve,
                          stream);
    if (rc) return rc;
    return labels_up2_launch(lc, c.Wc, c.Hc, c.sc.Q[0], c.sc.vmin[0], c.sc.vmin[1], W, H, space->Q[0], space->Q[1],
                             space->vmin[0], space->vmin[1], labels, st)
               ? EDP_ERR_CUDA
               : EDP_OK;
}

int edp_net_features_labels(const uint8_t *I0, const uint8_t *I1, const int32_t *labels, int W, int H, int pitch,
                            const edp_label_space *space, const edp_params *params, float scale, void *x,
                            edp_stream_t stream) {
    if (!I0 || !I1 || !labels || !x || !space || !params || W < 1 || H < 1 || pitch < W) return EDP_ERR_INVALID_ARG;
    if (space->R != 2 || space->step[0] != 1 || space->step[1] != 1 || !(scale > 0.f) || params->cmax < 1)
        return EDP_ERR_INVALID_ARG;
    return net_features_lab_launch(I0, I1, labels, W, H, pitch, space->Q[0], space->Q[1], space->vmin[0],
                                   space->vmin[1], params->l2, params->cmax, scale, x, (cudaStream_t)stream)
               ? EDP_ERR_CUDA
               : EDP_OK;
}

int edp_net_centres_residual(const float *out, const int32_t *base, int n, const edp_label_space *space,
                             int min_shift, int32_t *centre, edp_stream_t stream) {
    if (!out || !base || !centre || !space || n < 1 || space->R != 2 || min_shift < 0) return EDP_ERR_INVALID_ARG;
    return net_centres_base_launch(out, base, n, space->Q[0], space->Q[1], min_shift, centre, (cudaStream_t)stream)
               ? EDP_ERR_CUDA
               : EDP_OK;
}

int edp_window_edge_count(const int32_t *labels, const int32_t *centre, int n, int win,
                          const edp_label_space *space, int64_t *count, edp_stream_t stream) {
    if (!labels || !centre || !count || !space || n < 1 || space->R != 2) return EDP_ERR_INVALID_ARG;
    if (win < 1 || (win & 1) == 0 || win > space->Q[0] || win > space->Q[1]) return EDP_ERR_INVALID_ARG;
    return window_edge_count_launch(labels, centre, n, win, space->Q[0], space->Q[1],
                                    reinterpret_cast<unsigned long long *>(count), (cudaStream_t)stream)
               ? EDP_ERR_CUDA
               : EDP_OK;
}

int edp_net_targets(const int32_t *labels, const int32_t *base, int n, const edp_label_space *space, float *target,
                    edp_stream_t stream) {
    if (!labels || !target || !space || n < 1 || space->R != 2) return EDP_ERR_INVALID_ARG;
    return net_targets_launch(labels, base, n, space->Q[0], space->Q[1], target, (cudaStream_t)stream)
               ? EDP_ERR_CUDA
               : EDP_OK;
}

int edp_get_device_status(const void *ws, size_t ws_bytes, int *status, edp_stream_t stream) {
    if (!ws || !status || ws_bytes < kHeader) return EDP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cuda_status(cudaStreamSynchronize(st));
    if (rc) return rc;
    return cuda_status(cudaMemcpy(status, ws, sizeof(int), cudaMemcpyDeviceToHost));
}

}  // extern "C"
