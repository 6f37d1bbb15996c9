// rh15d_host.cu -- the C ABI (include/rh15d.h): context, atom tables,
// wavelength grid, column storage, launches.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "rh15d_ckpt.h"
#include "rh15d_internal.h"

using namespace rh;

namespace {

struct HostTrans {
    int l, u, kind, sub, prd = 0;
    double nu0, f, A, Blu, Bul, a_top, a_bot, qwing, alpha0, ratio, nu_lo, nu_hi;
    int nlam;
};

struct HostAtom {
    int nlev = 0, nline = 0, ncont = 0, ntr = 0, nmu = 0;
    double E[RH_MAXLEV], g[RH_MAXLEV];
    double mass = 0, T_ref = 0, floor_e = 0;
    std::vector<HostTrans> tr;
    std::vector<double> nu;                 // grid, band order
    std::vector<int> owner;                 // band transition of each point
    std::vector<std::vector<int>> act;      // active transitions per point
    std::vector<std::vector<double>> wq;    // quadrature weight of each active transition
    // tiles
    int ntile = 0, npad = 0;
    std::vector<int> lane_point;            // grid index of each padded lane, -1 padding
    std::vector<std::vector<int>> tile_union;
    double mu[RH_MAXMU], wmu[RH_MAXMU];
    // spontaneous-recombination sums of the start solutions: per transition
    // its continuum points (frequency, 4 pi w (2 h nu^3/c^2) alpha / (h nu))
    std::vector<int> sp_off;
    std::vector<double> sp_nu, sp_ce;
    // partial redistribution: PRD point of each padded lane (-1: none), and
    // per PRD point (PRD lines in order, frequency order) frequency and weight
    std::vector<int> lane_prd;
    std::vector<double> prd_nu, prd_w;
};

}  // namespace

struct rh_ctx {
    int dev = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int nsm = 0;
    std::string err;
    bool have_atom = false;
    HostAtom ha;
    DevAtom da;
    std::vector<double> lane_master;        // unscaled lane table, [kLaneFields][npad]
    void *lane_d = nullptr;                 // device lane table in the current precision/scale
    int lane_prec = -1;
    double lane_nref = 0;
    float4 *vtab_d = nullptr;
    float4 *dtab_d = nullptr;               // FP32 dispersion-function coefficient table
    // columns
    int64_t ncol = 0;
    int ndep = 0;
    double nref = 1.0;
    ColumnArrays ca{};
    double *nghist = nullptr;
    size_t nghist_cap = 0;
    int *queue = nullptr;
    long long *badidx = nullptr;
    int *colidx = nullptr;
    int64_t colidx_cap = 0;
    // learned initial guess
    rh::Mlp *mlp = nullptr;
    int mlp_ndep = 0;
    int mlp_hidden = 0, mlp_nhidden = 0;
    float *feat = nullptr, *tgt = nullptr, *lnb = nullptr;
    int64_t feat_cap = 0;
    int *idx_d = nullptr;
    int64_t idx_cap = 0;
    int *nfb_d = nullptr;
    double *loss_d = nullptr;
    // rh_solve: device counters and the captured sequence
    int *solve_cnt = nullptr;                   // [RH_MAX_RERUN] columns selected for each re-run pass
    unsigned long long *solve_it = nullptr;     // [1 + RH_MAX_RERUN] formal solutions of each pass
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned char> gkey;            // what the captured graph was built from
    int glaunches = 0;
    cudaEvent_t pass_ev[1 + RH_MAX_RERUN] = {};   // end of each pass (recorded inside the sequence)
    // partial redistribution: device tables and per-block scratch
    int *lane_prd_d = nullptr;
    double *prd_nu_d = nullptr, *prd_w_d = nullptr;
    void *prd_scr = nullptr;
    size_t prd_cap = 0;
    void *phic = nullptr;           // per-block profile cache of the column kernel
    size_t phic_cap = 0;
    // start solutions: device copy of the continuum point lists
    int *sp_off_d = nullptr;
    double *sp_nu_d = nullptr, *sp_ce_d = nullptr;
    // rh_autotune: chosen launch shape per precision (0: none)
    int tuned_bw[2] = {0, 0}, tuned_ctas[2] = {0, 0};
};

namespace {

int fail(rh_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(c, RH_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
void dfree(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

void drop_graph(rh_ctx *c)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    c->gkey.clear();
}

void free_columns(rh_ctx *c)
{
    drop_graph(c);
    dfree(c->ca.z);
    dfree(c->ca.T);
    dfree(c->ca.nH);
    dfree(c->ca.vz);
    dfree(c->ca.ne);
    dfree(c->ca.np);
    dfree(c->ca.nstar);
    dfree(c->ca.pops);
    dfree(c->ca.Crate);
    dfree(c->ca.dmax);
    dfree(c->ca.iters);
    dfree(c->ca.status);
    c->ncol = 0;
    c->ca.ncol = 0;
}

// Gauss-Legendre nodes/weights on (0,1) (weights sum to 1), Newton on P_n.
void gauss_legendre_unit(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int iter = 0; iter < 100; ++iter) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2 * j - 1) * z * p1 - (j - 1) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            double pn = n == 1 ? z : p1;
            double pm = n == 1 ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-15) {
                // one more evaluation of the derivative at the root
                p0 = 1.0;
                p1 = z;
                for (int j = 2; j <= n; ++j) {
                    double p2 = ((2 * j - 1) * z * p1 - (j - 1) * p0) / j;
                    p0 = p1;
                    p1 = p2;
                }
                pn = n == 1 ? z : p1;
                pm = n == 1 ? 1.0 : p0;
                dp = n * (z * pn - pm) / (z * z - 1.0);
                break;
            }
        }
        x[n - 1 - i] = 0.5 * (1.0 + z);
        w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

int build_atom(rh_ctx *c, const rh_atom_desc *d)
{
    HostAtom a;
    if (!d) return fail(c, RH_EINVAL, "desc is NULL");
    if (d->nlev < 2 || d->nlev > RH_MAXLEV) return fail(c, RH_EINVAL, "nlev must be in 2..%d", RH_MAXLEV);
    if (d->nline < 0 || d->ncont < 0 || d->nline + d->ncont < 1 || d->nline + d->ncont > RH_MAXTR)
        return fail(c, RH_EINVAL, "nline + ncont must be in 1..%d", RH_MAXTR);
    if (d->nmu < 1 || d->nmu > 8) return fail(c, RH_EINVAL, "nmu must be in 1..8");
    if (!(d->mass_amu > 0) || !(d->T_ref > 0) || !(d->metal_floor >= 0))
        return fail(c, RH_EINVAL, "mass_amu, T_ref must be > 0 and metal_floor >= 0");
    a.nlev = d->nlev;
    a.nline = d->nline;
    a.ncont = d->ncont;
    a.ntr = d->nline + d->ncont;
    a.nmu = d->nmu;
    a.mass = d->mass_amu * kAmu;
    a.T_ref = d->T_ref;
    a.floor_e = d->metal_floor;
    for (int i = 0; i < a.nlev; ++i) {
        a.E[i] = d->E_J[i];
        a.g[i] = d->g[i];
        if (!(a.g[i] > 0) || !std::isfinite(a.E[i])) return fail(c, RH_EINVAL, "level %d: bad E or g", i);
    }
    const int ic = a.nlev - 1;
    for (int i = 0; i < ic; ++i)
        if (!(a.E[ic] > a.E[i])) return fail(c, RH_EINVAL, "level %d lies above the continuum", i);
    for (int t = 0; t < d->nline; ++t) {
        HostTrans h{};
        h.l = d->line_l[t];
        h.u = d->line_u[t];
        if (h.l < 0 || h.u >= ic || h.l >= h.u) return fail(c, RH_EINVAL, "line %d: levels out of range", t);
        if (d->line_nlambda[t] < 2) return fail(c, RH_EINVAL, "line %d: line_nlambda < 2", t);
        if (!(d->line_f[t] > 0) || !(d->line_qwing[t] > 0) || !(d->line_a_top[t] > 0) || !(d->line_a_bot[t] > 0) ||
            d->line_a_top[t] > 0.05 || d->line_a_bot[t] > 0.05)
            return fail(c, RH_EINVAL, "line %d: f, qwing must be > 0 and damping in (0, 0.05]", t);
        h.kind = 0;
        h.sub = t;
        h.prd = (d->line_prd && d->line_prd[t]) ? 1 : 0;
        h.nu0 = (a.E[h.u] - a.E[h.l]) / kH;
        if (!(h.nu0 > 0)) return fail(c, RH_EINVAL, "line %d: upper level not above lower", t);
        h.f = d->line_f[t];
        h.A = 2.0 * kPi * kQ * kQ * h.nu0 * h.nu0 / (kEps0 * kMe * kC * kC * kC) * (a.g[h.l] / a.g[h.u]) * h.f;
        h.Bul = h.A * kC * kC / (2.0 * kH * h.nu0 * h.nu0 * h.nu0);
        h.Blu = h.Bul * a.g[h.u] / a.g[h.l];
        h.a_top = d->line_a_top[t];
        h.a_bot = d->line_a_bot[t];
        h.qwing = d->line_qwing[t];
        h.nlam = d->line_nlambda[t];
        double dnu = h.nu0 / kC * std::sqrt(2.0 * kK * a.T_ref / a.mass);
        h.nu_lo = h.nu0 - h.qwing * dnu;
        h.nu_hi = h.nu0 + h.qwing * dnu;
        a.tr.push_back(h);
    }
    for (int q = 0; q < d->ncont; ++q) {
        HostTrans h{};
        h.l = d->cont_l[q];
        h.u = ic;
        if (h.l < 0 || h.l >= ic) return fail(c, RH_EINVAL, "continuum %d: lower level out of range", q);
        if (d->cont_nlambda[q] < 2) return fail(c, RH_EINVAL, "continuum %d: cont_nlambda < 2", q);
        if (!(d->cont_ratio[q] > 1.0) || !(d->cont_alpha0[q] > 0))
            return fail(c, RH_EINVAL, "continuum %d: ratio must exceed 1 and alpha0 be > 0", q);
        h.kind = 1;
        h.sub = q;
        h.nu0 = (a.E[ic] - a.E[h.l]) / kH;
        h.alpha0 = d->cont_alpha0[q];
        h.ratio = d->cont_ratio[q];
        h.nlam = d->cont_nlambda[q];
        h.nu_lo = h.nu0;
        h.nu_hi = h.nu0 * h.ratio;
        a.tr.push_back(h);
    }
    gauss_legendre_unit(a.nmu, a.mu, a.wmu);
    // grid: bands in transition order
    const double beta = 5.0;
    for (int t = 0; t < a.ntr; ++t) {
        const HostTrans &h = a.tr[t];
        for (int j = 0; j < h.nlam; ++j) {
            double nu;
            if (h.kind == 0) {
                double s = -1.0 + 2.0 * j / (h.nlam - 1);
                double dnu = h.nu0 / kC * std::sqrt(2.0 * kK * a.T_ref / a.mass);
                nu = h.nu0 + h.qwing * std::sinh(beta * s) / std::sinh(beta) * dnu;
            } else {
                nu = h.nu0 * std::pow(h.ratio, (double)j / (h.nlam - 1));
            }
            a.nu.push_back(nu);
            a.owner.push_back(t);
        }
    }
    const size_t np = a.nu.size();
    a.act.resize(np);
    a.wq.resize(np);
    for (size_t i = 0; i < np; ++i) {
        for (int t = 0; t < a.ntr; ++t) {
            const HostTrans &h = a.tr[t];
            bool in = t == a.owner[i] ||
                      (a.nu[i] >= h.nu_lo * (1 - 1e-13) && a.nu[i] <= h.nu_hi * (1 + 1e-13));
            if (in) a.act[i].push_back(t);
        }
        a.wq[i].assign(a.act[i].size(), 0.0);
    }
    // trapezoid weights in frequency per transition over its active points
    for (int t = 0; t < a.ntr; ++t) {
        std::vector<std::pair<double, std::pair<size_t, size_t>>> pts;
        for (size_t i = 0; i < np; ++i)
            for (size_t s = 0; s < a.act[i].size(); ++s)
                if (a.act[i][s] == t) pts.push_back({a.nu[i], {i, s}});
        std::sort(pts.begin(), pts.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
        for (size_t j = 0; j < pts.size(); ++j) {
            double lo = j > 0 ? pts[j - 1].first : pts[j].first;
            double hi = j + 1 < pts.size() ? pts[j + 1].first : pts[j].first;
            a.wq[pts[j].second.first][pts[j].second.second] = 0.5 * (hi - lo);
        }
    }
    // tiles of 32 lanes within each band; a tile is closed (and padded) when it
    // is full or when the next point would bring more than RH_KMAX transitions
    // into the tile's union
    size_t p0 = 0;
    for (int t = 0; t < a.ntr; ++t) {
        int n = a.tr[t].nlam;
        std::vector<int> lanes, un;
        auto flush = [&]() {
            if (lanes.empty()) return;
            for (int l = 0; l < 32; ++l) a.lane_point.push_back(l < (int)lanes.size() ? lanes[l] : -1);
            std::sort(un.begin(), un.end());
            a.tile_union.push_back(un);
            lanes.clear();
            un.clear();
        };
        for (int j = 0; j < n; ++j) {
            const int gi = (int)(p0 + j);
            if ((int)a.act[gi].size() > RH_KMAX)
                return fail(c, RH_EINVAL, "%zu transitions overlap at one wavelength (max %d)", a.act[gi].size(),
                            RH_KMAX);
            std::vector<int> nu2 = un;
            for (int tt : a.act[gi])
                if (std::find(nu2.begin(), nu2.end(), tt) == nu2.end()) nu2.push_back(tt);
            if ((int)nu2.size() > RH_KMAX || lanes.size() == 32) {
                flush();
                nu2 = a.act[gi];
            }
            lanes.push_back(gi);
            un = nu2;
        }
        flush();
        p0 += n;
    }
    a.ntile = (int)a.tile_union.size();
    a.npad = a.ntile * 32;
    if (a.ntile > RH_MAXTILE) return fail(c, RH_EINVAL, "grid needs %d tiles (max %d)", a.ntile, RH_MAXTILE);

    // device atom
    DevAtom &da = c->da;
    memset(&da, 0, sizeof da);
    da.nlev = a.nlev;
    da.ntr = a.ntr;
    da.nline = a.nline;
    da.ncont = a.ncont;
    da.ntile = a.ntile;
    da.nmu = a.nmu;
    da.mass = a.mass;
    da.metal_floor = a.floor_e;
    for (int i = 0; i < ic; ++i) {
        da.lev_chi[i] = a.E[ic] - a.E[i];
        da.lev_g2[i] = a.g[i] / (2.0 * a.g[ic]);
    }
    for (int m = 0; m < a.nmu; ++m) {
        da.mu[m] = a.mu[m];
        da.wmu[m] = a.wmu[m];
        da.muf[m] = (float)a.mu[m];
        da.wm2f[m] = (float)(0.5 * a.wmu[m]);
        da.imuf[m] = (float)(1.0 / a.mu[m]);
    }
    for (int t = 0; t < a.ntr; ++t) {
        const HostTrans &h = a.tr[t];
        DevTrans &dt = da.tr[t];
        dt.l = h.l;
        dt.u = h.u;
        dt.kind = h.kind;
        dt.sub = h.sub;
        dt.nu0 = h.nu0;
        dt.A = h.A;
        dt.Blu = h.Blu;
        dt.Bul = h.Bul;
        dt.alpha0 = h.alpha0;
        dt.f = h.f;
        dt.ln_atop = h.kind == 0 ? std::log(h.a_top) : 0.0;
        dt.ln_abot = h.kind == 0 ? std::log(h.a_bot) : 0.0;
    }
    int acc = 0, nmap = 0;
    for (int b = 0; b < a.ntile; ++b) {
        const std::vector<int> &un = a.tile_union[b];
        int K = (int)un.size();
        DevTile &tl = da.tile[b];
        tl.K = K;
        for (int j = 0; j < K; ++j) tl.t[j] = un[j];
        tl.acc_off = acc;
        tl.m = K * (K + 1);
        auto add = [&](int accj, int row, int col, int sign) -> bool {
            if (row == col) return true;
            if (nmap >= RH_MAXMAP) return false;
            da.map_acc[nmap] = (int16_t)(acc + accj);
            da.map_row[nmap] = (int8_t)row;
            da.map_col[nmap] = (int8_t)col;
            da.map_sign[nmap] = (int8_t)sign;
            ++nmap;
            return true;
        };
        bool ok = true;
        for (int j = 0; j < K; ++j) {
            const HostTrans &h = a.tr[un[j]];
            ok &= add(j, h.u, h.l, +1);        // upward rate l -> u
            ok &= add(K + j, h.l, h.u, +1);    // downward rate u -> l (with the self cross term)
        }
        int idx = 2 * K;
        for (int j = 0; j < K; ++j)
            for (int j2 = 0; j2 < K; ++j2) {
                if (j2 == j) continue;
                const HostTrans &h = a.tr[un[j]], &h2 = a.tr[un[j2]];
                ok &= add(idx, h.l, h2.u, -1);
                ok &= add(idx, h.u, h2.u, +1);
                ++idx;
            }
        if (!ok) return fail(c, RH_EINVAL, "rate-matrix map exceeds %d entries", RH_MAXMAP);
        acc += tl.m;
    }
    da.macc = acc;
    da.nmap = nmap;
    // profile-cache rows: one per line slot of every tile
    da.nphi = 0;
    for (int b = 0; b < a.ntile; ++b) {
        DevTile &tl = da.tile[b];
        for (int j = 0; j < RH_KMAX; ++j) tl.phi[j] = -1;
        for (int j = 0; j < tl.K; ++j)
            if (a.tr[tl.t[j]].kind == 0) {
                da.phi_tile[da.nphi] = (int16_t)b;
                da.phi_j[da.nphi] = (int8_t)j;
                tl.phi[j] = da.nphi++;
            }
    }
    // partial redistribution
    {
        int np_lines = 0;
        for (int t = 0; t < a.ntr; ++t) np_lines += a.tr[t].prd;
        if (np_lines > RH_MAXPRD) return fail(c, RH_EINVAL, "at most %d PRD lines", RH_MAXPRD);
        int pacc = 0;
        for (int b = 0; b < a.ntile; ++b) {
            DevTile &tl = da.tile[b];
            tl.prd_slot = -1;
            for (int j = 0; j < tl.K; ++j)
                if (a.tr[tl.t[j]].prd) {
                    if (tl.prd_slot >= 0) return fail(c, RH_EINVAL, "two PRD lines overlap in wavelength");
                    tl.prd_slot = j;
                }
            tl.pacc_off = pacc;
            if (np_lines) pacc += 2 * tl.K;
        }
        da.pacc = pacc;
        std::vector<int> gi2lane(a.nu.size(), -1);
        for (int p = 0; p < a.npad; ++p)
            if (a.lane_point[p] >= 0) gi2lane[a.lane_point[p]] = p;
        a.lane_prd.assign(a.npad, -1);
        a.prd_nu.clear();
        a.prd_w.clear();
        da.nprd = 0;
        da.prd_off[0] = 0;
        da.prd_koff[0] = 0;
        for (int t = 0; t < a.ntr; ++t) {
            if (!a.tr[t].prd) continue;
            std::vector<std::pair<double, int>> pts;
            for (size_t gi = 0; gi < a.nu.size(); ++gi) {
                auto it = std::find(a.act[gi].begin(), a.act[gi].end(), t);
                if (it != a.act[gi].end()) pts.push_back({a.nu[gi], (int)gi});
            }
            std::sort(pts.begin(), pts.end());
            const int q = da.nprd++;
            da.prd_t[q] = t;
            for (auto &pr : pts) {
                const int gi = pr.second;
                const int pp = (int)a.prd_nu.size();
                if (pp >= RH_MAXPRDPT) return fail(c, RH_EINVAL, "more than %d PRD wavelength points", RH_MAXPRDPT);
                if (a.lane_prd[gi2lane[gi]] >= 0) return fail(c, RH_EINVAL, "two PRD lines share a wavelength point");
                a.lane_prd[gi2lane[gi]] = pp;
                a.prd_nu.push_back(pr.first);
                auto it = std::find(a.act[gi].begin(), a.act[gi].end(), t);
                a.prd_w.push_back(a.wq[gi][it - a.act[gi].begin()]);
            }
            const int npq = (int)pts.size();
            if (npq < 2) return fail(c, RH_EINVAL, "a PRD line needs at least two wavelength points");
            da.prd_off[q + 1] = da.prd_off[q] + npq;
            da.prd_koff[q + 1] = da.prd_koff[q] + npq * npq;
        }
        da.npp = (int)a.prd_nu.size();
    }
    // processing order: tiles with more transitions (costlier) first, line tiles before continua
    {
        std::vector<int> ord(a.ntile);
        for (int b = 0; b < a.ntile; ++b) ord[b] = b;
        auto cost = [&](int b) {
            int cst = 0;
            for (int t : a.tile_union[b]) cst += a.tr[t].kind == 0 ? 4 : 1;
            return cst;
        };
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cost(x) > cost(y); });
        for (int b = 0; b < a.ntile; ++b) da.order[b] = (int16_t)ord[b];
    }

    // lane master table (unscaled)
    const int F = kLaneFields;
    c->lane_master.assign((size_t)F * a.npad, 0.0);
    auto LM = [&](int f, int p) -> double & { return c->lane_master[(size_t)f * a.npad + p]; };
    for (int b = 0; b < a.ntile; ++b) {
        const std::vector<int> &un = a.tile_union[b];
        int first = -1;
        for (int l = 0; l < 32; ++l)
            if (a.lane_point[b * 32 + l] >= 0) {
                first = a.lane_point[b * 32 + l];
                break;
            }
        for (int l = 0; l < 32; ++l) {
            int p = b * 32 + l;
            int gi = a.lane_point[p];
            double nu = a.nu[gi >= 0 ? gi : first];
            LM(kLaneNu, p) = nu;
            LM(kLaneHm, p) = hminus_sigma(kC / nu);
            LM(kLaneNu3, p) = std::pow(1e15 / nu, 3);
            LM(kLaneTw, p) = 2.0 * kH * nu * nu * nu / (kC * kC);
            if (gi < 0) continue;
            for (size_t j = 0; j < un.size(); ++j) {
                int t = un[j];
                auto it = std::find(a.act[gi].begin(), a.act[gi].end(), t);
                if (it == a.act[gi].end()) continue;
                double w = a.wq[gi][it - a.act[gi].begin()];
                const HostTrans &h = a.tr[t];
                int f0 = RH_NLANEF * (int)j;
                if (h.kind == 0) {
                    double h4 = kH * nu / (4.0 * kPi);
                    LM(f0 + 0, p) = w * h.Blu;
                    LM(f0 + 1, p) = h4 * h.Blu;
                    LM(f0 + 2, p) = h4 * h.A;
                    LM(f0 + 3, p) = 2.0 * kH * h.nu0 * h.nu0 * h.nu0 / (kC * kC);
                    LM(f0 + 4, p) = kC * ((nu - h.nu0) / h.nu0);   // nu - nu0 is exact (Sterbenz)
                    LM(f0 + 5, p) = kC / (kSqrtPi * h.nu0);
                    LM(f0 + 6, p) = a.g[h.l] / a.g[h.u];
                } else {
                    double r = h.nu0 / nu;
                    double alpha = h.alpha0 * r * r * r;
                    double tw = 2.0 * kH * nu * nu * nu / (kC * kC);
                    LM(f0 + 0, p) = 4.0 * kPi * w * alpha / (kH * nu);
                    LM(f0 + 1, p) = alpha;
                    LM(f0 + 2, p) = tw * alpha;
                    LM(f0 + 3, p) = tw;
                }
            }
        }
    }
    a.sp_off.assign(1, 0);
    for (int t = 0; t < a.ntr; ++t) {
        const HostTrans &h = a.tr[t];
        if (h.kind != 0) {
            for (size_t gi = 0; gi < a.nu.size(); ++gi) {
                auto it = std::find(a.act[gi].begin(), a.act[gi].end(), t);
                if (it == a.act[gi].end()) continue;
                const double nu = a.nu[gi], w = a.wq[gi][it - a.act[gi].begin()];
                const double r = h.nu0 / nu, alpha = h.alpha0 * r * r * r;
                const double tw = 2.0 * kH * nu * nu * nu / (kC * kC);
                a.sp_nu.push_back(nu);
                a.sp_ce.push_back(4.0 * kPi * w * tw * alpha / (kH * nu));
            }
        }
        a.sp_off.push_back((int)a.sp_nu.size());
    }
    c->ha = std::move(a);
    return RH_OK;
}

// upload the lane table in precision prec with populations scaled by 1/nref
int ensure_lane(rh_ctx *c, int prec)
{
    if (c->lane_d && c->lane_prec == prec && c->lane_nref == c->nref) return RH_OK;
    dfree(c->lane_d);
    const int F = kLaneFields, np = c->ha.npad;
    std::vector<double> v = c->lane_master;
    for (int j = 0; j < RH_KMAX; ++j)
        for (int f : {1, 2})
            for (int p = 0; p < np; ++p) v[(size_t)(RH_NLANEF * j + f) * np + p] *= c->nref;
    size_t n = (size_t)F * np;
    if (prec == 1) {
        std::vector<float> h(n);
        for (size_t i = 0; i < n; ++i) h[i] = (float)v[i];
        CK(cudaMalloc(&c->lane_d, n * sizeof(float)));
        CK(cudaMemcpy(c->lane_d, h.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        CK(cudaMalloc(&c->lane_d, n * sizeof(double)));
        CK(cudaMemcpy(c->lane_d, v.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    }
    c->lane_prec = prec;
    c->lane_nref = c->nref;
    return RH_OK;
}

// PRD tables and the per-block scratch of the column kernel (as many blocks
// as the Ng history: 4 per SM)
int ensure_prd(rh_ctx *c, int precision)
{
    if (!c->da.nprd) return RH_OK;
    const HostAtom &a = c->ha;
    if (!c->lane_prd_d) {
        CK(cudaMalloc(&c->lane_prd_d, a.lane_prd.size() * sizeof(int)));
        CK(cudaMalloc(&c->prd_nu_d, a.prd_nu.size() * sizeof(double)));
        CK(cudaMalloc(&c->prd_w_d, a.prd_w.size() * sizeof(double)));
        CK(cudaMemcpy(c->lane_prd_d, a.lane_prd.data(), a.lane_prd.size() * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->prd_nu_d, a.prd_nu.data(), a.prd_nu.size() * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->prd_w_d, a.prd_w.data(), a.prd_w.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    const size_t want = mali_prd_bytes_per_block(c->da, c->ndep, precision) * (size_t)c->nsm * 4;
    if (c->prd_cap < want) {
        drop_graph(c);
        dfree(c->prd_scr);
        c->prd_cap = 0;
        CK(cudaMalloc(&c->prd_scr, want));
        c->prd_cap = want;
    }
    return RH_OK;
}

// Profile cache of the column kernel (as many blocks as the Ng history: 4 per SM)
int ensure_phic(rh_ctx *c, int precision)
{
    const size_t want = mali_phic_bytes_per_block(c->da, c->ndep, precision) * (size_t)c->nsm * 4;
    if (want && c->phic_cap < want) {
        drop_graph(c);
        dfree(c->phic);
        c->phic = nullptr;
        c->phic_cap = 0;
        CK(cudaMalloc(&c->phic, want));
        c->phic_cap = want;
    }
    return RH_OK;
}

void set_phic(const rh_ctx *c, IterLaunch &il)
{
    il.phic = c->phic;
    il.phic_cap = c->phic_cap;
}

void set_prd(const rh_ctx *c, IterLaunch &il, double eps0, int hybrid)
{
    il.prd_eps0 = eps0;
    il.prd_hybrid = hybrid;
    il.lane_prd = c->lane_prd_d;
    il.prd_nu = c->prd_nu_d;
    il.prd_w = c->prd_w_d;
    il.prd_scr = c->prd_scr;
    il.prd_cap = c->prd_cap;
}

int ensure_start_tables(rh_ctx *c)
{
    if (c->sp_off_d) return RH_OK;
    const HostAtom &a = c->ha;
    const size_t np = std::max<size_t>(1, a.sp_nu.size());
    CK(cudaMalloc(&c->sp_off_d, a.sp_off.size() * sizeof(int)));
    CK(cudaMalloc(&c->sp_nu_d, np * sizeof(double)));
    CK(cudaMalloc(&c->sp_ce_d, np * sizeof(double)));
    CK(cudaMemcpy(c->sp_off_d, a.sp_off.data(), a.sp_off.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (!a.sp_nu.empty()) {
        CK(cudaMemcpy(c->sp_nu_d, a.sp_nu.data(), a.sp_nu.size() * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->sp_ce_d, a.sp_ce.data(), a.sp_ce.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    return RH_OK;
}

// per requested wavelength: its frequency and up to RH_SPEC_ACT active
// transitions with their constants (see launch_spectrum)
int spectrum_tables(rh_ctx *c, int64_t nlambda, const double *lambda_m, std::vector<double> &nu,
                    std::vector<int> &nact, std::vector<int> &act, std::vector<double> &spec)
{
    const HostAtom &a = c->ha;
    nu.assign(nlambda, 0.0);
    spec.assign((size_t)nlambda * RH_SPEC_ACT * RH_SPEC_F, 0.0);
    nact.assign(nlambda, 0);
    act.assign((size_t)nlambda * RH_SPEC_ACT, 0);
    for (int64_t j = 0; j < nlambda; ++j) {
        if (!(lambda_m[j] > 0) || !std::isfinite(lambda_m[j]))
            return fail(c, RH_EINVAL, "wavelength %lld is not positive", (long long)j);
        double f = kC / lambda_m[j];
        nu[j] = f;
        for (int t = 0; t < a.ntr; ++t) {
            const HostTrans &h = a.tr[t];
            if (!(f >= h.nu_lo * (1 - 1e-13) && f <= h.nu_hi * (1 + 1e-13))) continue;
            if (nact[j] >= RH_SPEC_ACT) return fail(c, RH_EINVAL, "more than %d transitions at one wavelength", RH_SPEC_ACT);
            int s = nact[j]++;
            act[j * RH_SPEC_ACT + s] = t;
            double *p = &spec[((size_t)j * RH_SPEC_ACT + s) * RH_SPEC_F];
            if (h.kind == 0) {
                double h4 = kH * f / (4.0 * kPi);
                p[0] = h4 * h.Blu;
                p[1] = h4 * h.A;
                p[2] = a.g[h.l] / a.g[h.u];
                p[3] = kC * ((f - h.nu0) / h.nu0);
                p[4] = kC / (kSqrtPi * h.nu0);
            } else {
                double r = h.nu0 / f;
                double alpha = h.alpha0 * r * r * r;
                p[0] = alpha;
                p[1] = 2.0 * kH * f * f * f / (kC * kC) * alpha;
            }
        }
    }
    return RH_OK;
}

__global__ void validate_kernel(int64_t ncol, int ndep, const double *z, const double *T, const double *ne,
                                const double *nH, const double *vz, unsigned long long *bad)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncol * ndep) return;
    int k = (int)(i % ndep);
    bool ok = isfinite(T[i]) && T[i] > 0 && isfinite(nH[i]) && nH[i] > 0 && isfinite(z[i]) && isfinite(vz[i]) &&
              (!ne || (isfinite(ne[i]) && ne[i] > 0));
    if (ok && k > 0) ok = z[i] < z[i - 1];
    if (!ok) atomicMin(bad, (unsigned long long)i);
}

// feature / target / prediction buffers for the loaded columns
int ensure_mlp_buffers(rh_ctx *c)
{
    const int64_t nin = 4LL * c->ndep, nout = (int64_t)c->da.nlev * c->ndep;
    if (c->feat_cap < c->ncol) {
        dfree(c->feat);
        dfree(c->tgt);
        dfree(c->lnb);
        CK(cudaMalloc(&c->feat, c->ncol * nin * sizeof(float)));
        CK(cudaMalloc(&c->tgt, c->ncol * nout * sizeof(float)));
        CK(cudaMalloc(&c->lnb, c->ncol * nout * sizeof(float)));
        c->feat_cap = c->ncol;
    }
    if (!c->nfb_d) CK(cudaMalloc(&c->nfb_d, sizeof(int)));
    if (!c->loss_d) CK(cudaMalloc(&c->loss_d, sizeof(double)));
    return RH_OK;
}

int ensure_idx(rh_ctx *c, int64_t n)
{
    if (n > c->idx_cap) {
        dfree(c->idx_d);
        CK(cudaMalloc(&c->idx_d, n * sizeof(int)));
        c->idx_cap = n;
    }
    return RH_OK;
}

}  // namespace

// ============================================================================
extern "C" {

int rh_surrogate_init(rh_ctx *c, int32_t hidden, int32_t nhidden, uint64_t seed)
{
    if (!c) return RH_EINVAL;
    drop_graph(c);   // network buffers may be (re)allocated
    if (!c->ncol) return fail(c, RH_ESTATE, "rh_surrogate_init: load columns first (the network size follows ndep)");
    if (hidden < 8 || hidden > 4096 || nhidden < 1 || nhidden > 8)
        return fail(c, RH_EINVAL, "rh_surrogate_init: hidden in 8..4096, nhidden in 1..8");
    cudaSetDevice(c->dev);
    if (c->mlp) mlp_destroy(c->mlp);
    c->mlp = nullptr;
    CK(mlp_create(&c->mlp, 4 * c->ndep, hidden, nhidden, c->da.nlev * c->ndep, seed));
    c->mlp_ndep = c->ndep;
    c->mlp_hidden = hidden;
    c->mlp_nhidden = nhidden;
    return RH_OK;
}

int64_t rh_surrogate_state_size(const rh_ctx *c) { return (c && c->mlp) ? mlp_state_size(c->mlp) : 0; }

int rh_surrogate_get_state(rh_ctx *c, float *out)
{
    if (!c || !out) return RH_EINVAL;
    if (!c->mlp) return fail(c, RH_ESTATE, "no surrogate");
    cudaSetDevice(c->dev);
    CK(mlp_get_state(c->mlp, out));
    return RH_OK;
}

int rh_surrogate_set_state(rh_ctx *c, const float *in)
{
    if (!c || !in) return RH_EINVAL;
    drop_graph(c);   // network buffers may be (re)allocated
    if (!c->mlp) return fail(c, RH_ESTATE, "no surrogate (rh_surrogate_init first)");
    for (int64_t i = 0; i < mlp_state_size(c->mlp); ++i)
        if (!std::isfinite(in[i])) return fail(c, RH_EINVAL, "surrogate state entry %lld is not finite", (long long)i);
    cudaSetDevice(c->dev);
    CK(mlp_set_state(c->mlp, in));
    return RH_OK;
}

int rh_surrogate_train(rh_ctx *c, const rh_train_opts *o, rh_train_stats *st)
{
    if (!c || !o) return RH_EINVAL;
    drop_graph(c);   // network buffers may be (re)allocated
    if (!c->mlp || c->mlp_ndep != c->ndep) return fail(c, RH_ESTATE, "rh_surrogate_train: no surrogate for these columns");
    if (o->epochs < 1 || o->batch < 1 || !(o->lr > 0) || !(o->beta1 >= 0 && o->beta1 < 1) ||
        !(o->beta2 >= 0 && o->beta2 < 1) || !(o->eps > 0))
        return fail(c, RH_EINVAL, "rh_surrogate_train: invalid options");
    cudaSetDevice(c->dev);
    std::vector<uint8_t> stt(c->ncol);
    CK(cudaMemcpy(stt.data(), c->ca.status, c->ncol, cudaMemcpyDeviceToHost));
    std::vector<int> rows;
    for (int64_t i = 0; i < c->ncol; ++i)
        if (stt[i] == RH_COL_CONVERGED) rows.push_back((int)i);
    if (rows.empty()) return fail(c, RH_ESTATE, "rh_surrogate_train: no converged columns to learn from");
    int r = ensure_mlp_buffers(c);
    if (r) return r;
    const int64_t nr = (int64_t)rows.size();
    r = ensure_idx(c, std::max<int64_t>(nr, o->batch));
    if (r) return r;
    const auto t0 = std::chrono::steady_clock::now();
    CK(mlp_features(c->ca, c->feat, c->st));
    CK(mlp_targets(c->ca, c->da.nlev, c->tgt, c->st));
    if (o->standardise) {
        CK(cudaMemcpyAsync(c->idx_d, rows.data(), nr * sizeof(int), cudaMemcpyHostToDevice, c->st));
        CK(mlp_set_standardisation(c->mlp, c->feat, c->idx_d, nr, c->st));
    }
    std::mt19937_64 rng(o->seed);
    const int64_t B = std::min<int64_t>(o->batch, nr);
    const int64_t per_epoch = nr / B;
    const int64_t total = per_epoch * o->epochs;
    rh_train_stats S{};
    int64_t step = 0;
    std::vector<int> perm(rows);
    for (int ep = 0; ep < o->epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        CK(cudaMemcpyAsync(c->idx_d, perm.data(), per_epoch * B * sizeof(int), cudaMemcpyHostToDevice, c->st));
        double esum = 0.0;
        for (int64_t b = 0; b < per_epoch; ++b, ++step) {
            CK(mlp_loss_grad(c->mlp, B, c->feat, c->tgt, c->idx_d + b * B, c->loss_d, c->st));
            double loss = 0.0;
            CK(cudaMemcpyAsync(&loss, c->loss_d, sizeof(double), cudaMemcpyDeviceToHost, c->st));
            float lr = (float)(o->lr * 0.5 * (1.0 + std::cos(3.14159265358979 * (double)step / (double)total)));
            CK(mlp_adam(c->mlp, lr, o->beta1, o->beta2, o->eps, c->st));
            CK(cudaStreamSynchronize(c->st));
            if (!std::isfinite(loss)) return fail(c, RH_ENOTCONV, "rh_surrogate_train: loss is not finite at step %lld",
                                                  (long long)step);
            esum += loss;
        }
        double em = esum / (double)per_epoch;
        if (ep == 0) S.loss_first_epoch = em;
        S.loss_last_epoch = em;
    }
    S.steps = step;
    S.samples = step * B;
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (st) *st = S;
    return RH_OK;
}

int rh_surrogate_loss_grad(rh_ctx *c, int64_t ncols, const int32_t *cols, double *loss_out, float *grad_out)
{
    if (!c || !cols || ncols < 1) return RH_EINVAL;
    drop_graph(c);   // network buffers may be (re)allocated
    if (!c->mlp || c->mlp_ndep != c->ndep) return fail(c, RH_ESTATE, "no surrogate for these columns");
    for (int64_t i = 0; i < ncols; ++i)
        if (cols[i] < 0 || cols[i] >= c->ncol) return fail(c, RH_EINVAL, "column index %d out of range", cols[i]);
    cudaSetDevice(c->dev);
    int r = ensure_mlp_buffers(c);
    if (r) return r;
    r = ensure_idx(c, ncols);
    if (r) return r;
    CK(mlp_features(c->ca, c->feat, c->st));
    CK(mlp_targets(c->ca, c->da.nlev, c->tgt, c->st));
    CK(cudaMemcpyAsync(c->idx_d, cols, ncols * sizeof(int), cudaMemcpyHostToDevice, c->st));
    CK(mlp_loss_grad(c->mlp, ncols, c->feat, c->tgt, c->idx_d, c->loss_d, c->st));
    double loss = 0.0;
    CK(cudaMemcpyAsync(&loss, c->loss_d, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (grad_out) {
        const int64_t np = mlp_nparams(c->mlp);
        CK(cudaMemcpyAsync(grad_out, mlp_grad(c->mlp), np * sizeof(float), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        for (int64_t i = np; i < mlp_state_size(c->mlp); ++i) grad_out[i] = 0.f;
    }
    CK(cudaStreamSynchronize(c->st));
    if (loss_out) *loss_out = loss;
    return RH_OK;
}

int rh_surrogate_predict(rh_ctx *c, float *lnb_out)
{
    if (!c || !lnb_out) return RH_EINVAL;
    drop_graph(c);   // network buffers may be (re)allocated
    if (!c->mlp || c->mlp_ndep != c->ndep) return fail(c, RH_ESTATE, "no surrogate for these columns");
    cudaSetDevice(c->dev);
    int r = ensure_mlp_buffers(c);
    if (r) return r;
    // prediction into lnb; the populations are restored afterwards
    double *save = nullptr;
    const size_t nv = (size_t)c->ncol * c->da.nlev * c->ndep;
    CK(cudaMalloc(&save, nv * 8));
    cudaError_t e = cudaMemcpyAsync(save, c->ca.pops, nv * 8, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = mlp_predict_apply(c->mlp, c->ca, c->da.nlev, c->feat, c->lnb, c->nfb_d, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ca.pops, save, nv * 8, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lnb_out, c->lnb, nv * 4, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    cudaFree(save);
    if (e != cudaSuccess) return fail(c, RH_ECUDA, "rh_surrogate_predict: %s", cudaGetErrorString(e));
    return RH_OK;
}

int rh_surrogate_save(rh_ctx *c, const char *path)
{
    if (!c || !path) return RH_EINVAL;
    if (!c->mlp) return fail(c, RH_ESTATE, "rh_surrogate_save: no surrogate");
    cudaSetDevice(c->dev);
    std::vector<float> st((size_t)mlp_state_size(c->mlp));
    CK(mlp_get_state(c->mlp, st.data()));
    CkptSizes z;
    z.nin = 4 * c->mlp_ndep;
    z.hidden = c->mlp_hidden;
    z.nhidden = c->mlp_nhidden;
    z.nout = c->da.nlev * c->mlp_ndep;
    if (ckpt_nparam(z) != (int64_t)st.size()) return fail(c, RH_EINVAL, "rh_surrogate_save: inconsistent network sizes");
    const char *why = ckpt_write(path, z, st.data(), (int64_t)st.size());
    if (why) return fail(c, RH_EINVAL, "rh_surrogate_save: %s: %s", path, why);
    return RH_OK;
}

int rh_surrogate_load(rh_ctx *c, const char *path)
{
    if (!c || !path) return RH_EINVAL;
    if (!c->ncol) return fail(c, RH_ESTATE, "rh_surrogate_load: load columns first (the network size follows ndep)");
    CkptSizes z;
    int64_t np = 0;
    std::vector<float> st;
    const char *why = ckpt_read(path, z, np, &st);
    if (why) return fail(c, RH_EINVAL, "rh_surrogate_load: %s: %s", path, why);
    if (z.nin != 4 * c->ndep || z.nout != c->da.nlev * c->ndep)
        return fail(c, RH_EINVAL, "rh_surrogate_load: the checkpoint is for %d inputs and %d outputs, the loaded "
                                  "columns need %d and %d", z.nin, z.nout, 4 * c->ndep, c->da.nlev * c->ndep);
    int r = rh_surrogate_init(c, z.hidden, z.nhidden, 0);
    if (r) return r;
    if (mlp_state_size(c->mlp) != np) return fail(c, RH_EINVAL, "rh_surrogate_load: state length mismatch");
    return rh_surrogate_set_state(c, st.data());
}

int rh_surrogate_file_info(const char *path, int32_t *sizes_out, int64_t *nparam_out, char *msg, size_t msg_len)
{
    if (msg && msg_len) msg[0] = 0;
    if (!path) return RH_EINVAL;
    CkptSizes z;
    int64_t np = 0;
    const char *why = ckpt_read(path, z, np, nullptr);
    if (why) {
        if (msg && msg_len) snprintf(msg, msg_len, "%s", why);
        return RH_EINVAL;
    }
    if (sizes_out) {
        sizes_out[0] = z.nin;
        sizes_out[1] = z.hidden;
        sizes_out[2] = z.nhidden;
        sizes_out[3] = z.nout;
    }
    if (nparam_out) *nparam_out = np;
    return RH_OK;
}

int rh_create(rh_ctx **out, int cuda_device, void *cuda_stream)
{
    if (!out) return RH_EINVAL;
    *out = nullptr;
    rh_ctx *c = new (std::nothrow) rh_ctx();
    if (!c) return RH_ENOMEM;
    c->dev = cuda_device;
    cudaError_t e = cudaSetDevice(cuda_device);
    if (e == cudaSuccess && cuda_stream) {
        c->st = (cudaStream_t)cuda_stream;
    } else if (e == cudaSuccess) {
        e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
        c->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, cuda_device);
    if (e == cudaSuccess) e = cudaMalloc(&c->queue, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->badidx, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        *out = c;
        c->err = std::string("rh_create: ") + cudaGetErrorString(e);
        return RH_ECUDA;
    }
    // coefficient table of the FP32 Voigt function, uniform in t = 1/(1+|v|)
    std::vector<float4> vt(RH_VT_N + 1);
    const double hh = 1.0 / RH_VT_N;
    for (int i = 0; i <= RH_VT_N; ++i) {
        if (i == 0) {
            vt[i] = make_float4(0.f, 0.f, 0.f, 0.f);   // v -> infinity: H1, H3 ~ t^2
            continue;
        }
        double t = i * hh, v = 1.0 / t - 1.0, h1, d1, h3, d3;
        voigt_coeffs(v, h1, d1, h3, d3);
        double dvdt = -1.0 / (t * t);
        vt[i] = make_float4((float)h1, (float)(hh * d1 * dvdt), (float)h3, (float)(hh * d3 * dvdt));
    }
    e = cudaMalloc(&c->vtab_d, (RH_VT_N + 1) * sizeof(float4));
    if (e == cudaSuccess) e = cudaMemcpy(c->vtab_d, vt.data(), (RH_VT_N + 1) * sizeof(float4), cudaMemcpyHostToDevice);
    // and of the FP32 dispersion function (L0 ~ t/sqrt(pi), L2 ~ t^3 as t -> 0)
    std::vector<float4> dt(RH_VT_N + 1);
    for (int i = 0; i <= RH_VT_N; ++i) {
        if (i == 0) {
            dt[i] = make_float4(0.f, (float)(hh / kSqrtPi), 0.f, 0.f);
            continue;
        }
        double t = i * hh, v = 1.0 / t - 1.0, l0, d0, l2, d2;
        dispersion_coeffs(v, l0, d0, l2, d2);
        double dvdt = -1.0 / (t * t);
        dt[i] = make_float4((float)l0, (float)(hh * d0 * dvdt), (float)l2, (float)(hh * d2 * dvdt));
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->dtab_d, (RH_VT_N + 1) * sizeof(float4));
    if (e == cudaSuccess) e = cudaMemcpy(c->dtab_d, dt.data(), (RH_VT_N + 1) * sizeof(float4), cudaMemcpyHostToDevice);
    *out = c;
    if (e != cudaSuccess) {
        c->err = std::string("rh_create: ") + cudaGetErrorString(e);
        return RH_ECUDA;
    }
    return RH_OK;
}

void rh_destroy(rh_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->dev);
    if (c->st) cudaStreamSynchronize(c->st);
    free_columns(c);
    dfree(c->lane_d);
    dfree(c->vtab_d);
    dfree(c->dtab_d);
    dfree(c->nghist);
    dfree(c->prd_scr);
    dfree(c->phic);
    dfree(c->queue);
    dfree(c->badidx);
    dfree(c->colidx);
    if (c->mlp) mlp_destroy(c->mlp);
    dfree(c->feat);
    dfree(c->tgt);
    dfree(c->lnb);
    dfree(c->idx_d);
    dfree(c->nfb_d);
    dfree(c->loss_d);
    dfree(c->solve_cnt);
    dfree(c->solve_it);
    dfree(c->sp_off_d);
    dfree(c->sp_nu_d);
    dfree(c->sp_ce_d);
    drop_graph(c);
    dfree(c->lane_prd_d);
    dfree(c->prd_nu_d);
    dfree(c->prd_w_d);
    for (cudaEvent_t &ev : c->pass_ev)
        if (ev) cudaEventDestroy(ev);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c;
}

const char *rh_last_error(const rh_ctx *c) { return c ? c->err.c_str() : "null context"; }

int rh_setup_atom(rh_ctx *c, const rh_atom_desc *d)
{
    if (!c) return RH_EINVAL;
    if (c->ncol) return fail(c, RH_ESTATE, "rh_setup_atom: columns are loaded; set the atom first");
    cudaSetDevice(c->dev);
    c->have_atom = false;
    int r = build_atom(c, d);
    if (r) return r;
    dfree(c->lane_d);
    dfree(c->sp_off_d);
    dfree(c->sp_nu_d);
    dfree(c->sp_ce_d);
    dfree(c->lane_prd_d);
    dfree(c->prd_nu_d);
    dfree(c->prd_w_d);
    c->lane_prec = -1;
    c->tuned_bw[0] = c->tuned_bw[1] = c->tuned_ctas[0] = c->tuned_ctas[1] = 0;
    drop_graph(c);
    c->have_atom = true;
    return RH_OK;
}

int64_t rh_nlambda(const rh_ctx *c) { return (c && c->have_atom) ? (int64_t)c->ha.nu.size() : 0; }

int rh_get_grid(const rh_ctx *c, double *nu_out)
{
    if (!c || !c->have_atom || !nu_out) return RH_EINVAL;
    memcpy(nu_out, c->ha.nu.data(), c->ha.nu.size() * sizeof(double));
    return RH_OK;
}

int rh_load_columns(rh_ctx *c, int64_t ncol, int32_t ndep, const double *z_m, const double *T_K,
                    const double *ne_m3, const double *nH_m3, const double *vz_ms, int32_t on_device)
{
    if (!c) return RH_EINVAL;
    if (!c->have_atom) return fail(c, RH_ESTATE, "rh_load_columns: no atom");
    if (ncol < 1 || ndep < 2 || ndep > 4096) return fail(c, RH_EINVAL, "need ncol >= 1 and 2 <= ndep <= 4096");
    if (!z_m || !T_K || !nH_m3 || !vz_ms) return fail(c, RH_EINVAL, "z, T, nH, vz must not be NULL");
    cudaSetDevice(c->dev);
    if (ndep != c->ndep) c->tuned_bw[0] = c->tuned_bw[1] = c->tuned_ctas[0] = c->tuned_ctas[1] = 0;
    free_columns(c);
    const int L = c->da.nlev;
    const size_t nd = (size_t)ncol * ndep;
    ColumnArrays &a = c->ca;
    a.ncol = ncol;
    a.ndep = ndep;
    CK(cudaMalloc(&a.z, nd * 8));
    CK(cudaMalloc(&a.T, nd * 8));
    CK(cudaMalloc(&a.nH, nd * 8));
    CK(cudaMalloc(&a.vz, nd * 8));
    CK(cudaMalloc(&a.ne, nd * 8));
    CK(cudaMalloc(&a.np, nd * 8));
    CK(cudaMalloc(&a.nstar, nd * L * 8));
    CK(cudaMalloc(&a.pops, nd * L * 8));
    CK(cudaMalloc(&a.Crate, nd * 2 * c->da.ntr * 8));
    CK(cudaMalloc(&a.dmax, ncol * 8));
    CK(cudaMalloc(&a.iters, ncol * 4));
    CK(cudaMalloc(&a.status, ncol));
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(a.z, z_m, nd * 8, kind, c->st));
    CK(cudaMemcpyAsync(a.T, T_K, nd * 8, kind, c->st));
    CK(cudaMemcpyAsync(a.nH, nH_m3, nd * 8, kind, c->st));
    CK(cudaMemcpyAsync(a.vz, vz_ms, nd * 8, kind, c->st));
    if (ne_m3) CK(cudaMemcpyAsync(a.ne, ne_m3, nd * 8, kind, c->st));
    CK(cudaMemsetAsync(a.iters, 0, ncol * 4, c->st));
    CK(cudaMemsetAsync(a.status, RH_COL_NOTRUN, ncol, c->st));
    CK(cudaMemsetAsync(a.dmax, 0, ncol * 8, c->st));
    unsigned long long bad0 = ~0ull;
    CK(cudaMemcpyAsync(c->badidx, &bad0, 8, cudaMemcpyHostToDevice, c->st));
    validate_kernel<<<(unsigned)((nd + 255) / 256), 256, 0, c->st>>>(ncol, ndep, a.z, a.T, ne_m3 ? a.ne : nullptr,
                                                                   a.nH, a.vz, (unsigned long long *)c->badidx);
    CK(cudaGetLastError());
    unsigned long long bad = 0;
    CK(cudaMemcpyAsync(&bad, c->badidx, 8, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (bad != ~0ull) {
        long long col = (long long)(bad / ndep), k = (long long)(bad % ndep);
        free_columns(c);
        return fail(c, RH_EINVAL,
                    "invalid input at column %lld depth %lld (need finite T, n_H, n_e > 0, finite v_z, z decreasing)",
                    col, k);
    }
    c->ncol = ncol;
    c->ndep = ndep;
    CK(launch_lte_setup(c->da, a, ne_m3 ? 1 : 0, c->st));
    CK(cudaStreamSynchronize(c->st));
    // reference density of the FP32 population scaling: a fixed constant, so
    // that a column's result does not depend on which other columns are
    // loaded (populations 1e-10 .. 1e25 m^-3 map to 1e-30 .. 1e5)
    c->nref = 1e20;
    return RH_OK;
}

int rh_iterate(rh_ctx *c, const rh_iter_opts *o, rh_iter_stats *st)
{
    if (!c) return RH_EINVAL;
    if (!c->ncol) return fail(c, RH_ESTATE, "rh_iterate: no columns loaded");
    if (!o) return fail(c, RH_EINVAL, "opts is NULL");
    if (o->maxiter < 1 || !(o->tol >= 0) || (o->ng_order != 0 && o->ng_order != 2) ||
        (o->ng_order == 2 && (o->ng_period < 1 || o->ng_delay < 0)) || (o->precision != 0 && o->precision != 1) ||
        (o->start < 0 || o->start > 4) || o->block_warps < 0 || o->block_warps > 8 ||
        (o->only_unconverged != 0 && o->only_unconverged != 1) || !std::isfinite(o->prd_eps0) ||
        (o->prd_hybrid != 0 && o->prd_hybrid != 1) || (o->formal != 0 && o->formal != 1))
        return fail(c, RH_EINVAL, "rh_iterate: invalid options");
    cudaSetDevice(c->dev);
    int start = o->start;
    int64_t fallback = 0;
    double guess_s = 0.0;
    float guess_ms = 0.f;
    if (start == 1) {
        if (!c->mlp || c->mlp_ndep != c->ndep)
            return fail(c, RH_ESTATE, "rh_iterate: start = 1 needs a surrogate for %d depths (rh_surrogate_init)",
                        c->ndep);
        if (o->only_unconverged)
            return fail(c, RH_EINVAL, "rh_iterate: start = 1 applies to all columns (only_unconverged = 0)");
        int r = ensure_mlp_buffers(c);
        if (r) return r;
        cudaEvent_t g0, g1;
        CK(cudaEventCreate(&g0));
        CK(cudaEventCreate(&g1));
        CK(cudaEventRecord(g0, c->st));
        CK(mlp_predict_apply(c->mlp, c->ca, c->da.nlev, c->feat, c->lnb, c->nfb_d, c->st));
        CK(cudaEventRecord(g1, c->st));
        int nfb = 0;
        CK(cudaMemcpyAsync(&nfb, c->nfb_d, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        cudaEventElapsedTime(&guess_ms, g0, g1);
        cudaEventDestroy(g0);
        cudaEventDestroy(g1);
        fallback = nfb;
        guess_s = guess_ms * 1e-3;
        start = 2;
    } else if (start == 3 || start == 4) {
        if (o->only_unconverged)
            return fail(c, RH_EINVAL, "rh_iterate: start = %d applies to all columns (only_unconverged = 0)", start);
        int r = ensure_start_tables(c);
        if (r) return r;
        cudaEvent_t g0, g1;
        CK(cudaEventCreate(&g0));
        CK(cudaEventCreate(&g1));
        CK(cudaEventRecord(g0, c->st));
        CK(launch_start(c->da, c->ca, start, c->sp_off_d, c->sp_nu_d, c->sp_ce_d, c->st));
        CK(cudaEventRecord(g1, c->st));
        CK(cudaEventSynchronize(g1));
        cudaEventElapsedTime(&guess_ms, g0, g1);
        cudaEventDestroy(g0);
        cudaEventDestroy(g1);
        guess_s = guess_ms * 1e-3;
        start = 2;
    }
    // work list: every column, or the columns not converged so far
    int64_t nwork = c->ncol;
    const int *colidx_d = nullptr;
    if (o->only_unconverged) {
        std::vector<uint8_t> st0(c->ncol);
        CK(cudaMemcpy(st0.data(), c->ca.status, c->ncol, cudaMemcpyDeviceToHost));
        std::vector<int> idx;
        for (int64_t i = 0; i < c->ncol; ++i)
            if (st0[i] != RH_COL_CONVERGED) idx.push_back((int)i);
        nwork = (int64_t)idx.size();
        if (nwork > c->colidx_cap) {
            dfree(c->colidx);
            CK(cudaMalloc(&c->colidx, nwork * sizeof(int)));
            c->colidx_cap = nwork;
        }
        if (nwork) CK(cudaMemcpy(c->colidx, idx.data(), nwork * sizeof(int), cudaMemcpyHostToDevice));
        colidx_d = c->colidx;
    }
    int r = ensure_lane(c, o->precision);
    if (r) return r;
    r = ensure_prd(c, o->precision);
    if (r) return r;
    r = ensure_phic(c, o->precision);
    if (r) return r;
    size_t per_block = mali_nghist_bytes_per_block(c->da, c->ndep);
    size_t want = per_block * (size_t)c->nsm * 4;
    if (c->nghist_cap < want) {
        dfree(c->nghist);
        c->nghist_cap = 0;
        CK(cudaMalloc(&c->nghist, want));
        c->nghist_cap = want;
    }
    IterLaunch il;
    il.precision = o->precision;
    il.formal = o->formal;
    il.persistent = o->persistent;
    il.block_warps = o->block_warps;
    il.maxiter = o->maxiter;
    il.ng_order = o->ng_order;
    il.ng_delay = o->ng_delay;
    il.ng_period = o->ng_period;
    il.start = start;
    il.tol = o->tol;
    il.crsw = o->crsw_init;
    il.nsm = c->nsm;
    il.colidx = colidx_d;
    il.nwork = nwork;
    if (o->block_warps == 0 && c->tuned_bw[o->precision]) {
        il.block_warps = c->tuned_bw[o->precision];
        il.ctas_per_sm = c->tuned_ctas[o->precision];
    }
    set_prd(c, il, o->prd_eps0, o->prd_hybrid);
    set_phic(c, il);
    float ms = 0;
    int grid = 0;
    char ebuf[256] = {0};
    if (nwork > 0) {
        cudaError_t e = launch_mali(c->da, c->ca, c->lane_d, c->ha.npad, c->vtab_d, c->nref, c->nghist,
                                    c->nghist_cap, c->queue, il, c->st, &ms, &grid, ebuf, sizeof ebuf);
        if (e != cudaSuccess)
            return fail(c, RH_ECUDA, "rh_iterate: %s%s%s", cudaGetErrorString(e), ebuf[0] ? ": " : "", ebuf);
    }
    std::vector<int32_t> it(c->ncol);
    std::vector<uint8_t> s(c->ncol);
    std::vector<double> dm(c->ncol);
    CK(cudaMemcpy(it.data(), c->ca.iters, c->ncol * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(s.data(), c->ca.status, c->ncol, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(dm.data(), c->ca.dmax, c->ncol * 8, cudaMemcpyDeviceToHost));
    rh_iter_stats S{};
    S.seconds = ms * 1e-3 + guess_s;
    S.guess_seconds = guess_s;
    S.guess_fallback_depths = fallback;
    S.n_processed = nwork;
    std::vector<char> done(c->ncol, o->only_unconverged ? 0 : 1);
    if (o->only_unconverged) {
        std::vector<int> idx(nwork);
        if (nwork) CK(cudaMemcpy(idx.data(), c->colidx, nwork * sizeof(int), cudaMemcpyDeviceToHost));
        for (int i : idx) done[i] = 1;
    }
    for (int64_t i = 0; i < c->ncol; ++i) {
        if (s[i] == RH_COL_CONVERGED) S.n_converged++;
        else if (s[i] == RH_COL_MAXITER) S.n_maxiter++;
        else S.n_failed++;
        if (done[i]) S.iterations_total += it[i];
        if (dm[i] > S.max_dn_final) S.max_dn_final = dm[i];   // NaN entries skipped
    }
    S.pts = (double)S.iterations_total * c->ndep * (double)c->ha.nu.size() * c->ha.nmu;
    if (st) *st = S;
    return (S.n_maxiter || S.n_failed) ? RH_ENOTCONV : RH_OK;
}

int rh_get_populations(rh_ctx *c, double *n_out, int32_t *iters, uint8_t *status, double *dmax, int32_t on_device)
{
    if (!c) return RH_EINVAL;
    if (!c->ncol) return fail(c, RH_ESTATE, "no columns loaded");
    cudaSetDevice(c->dev);
    CK(cudaStreamSynchronize(c->st));
    size_t nv = (size_t)c->ncol * c->ndep * c->da.nlev;
    if (n_out) CK(cudaMemcpy(n_out, c->ca.pops, nv * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    if (iters) CK(cudaMemcpy(iters, c->ca.iters, c->ncol * 4, cudaMemcpyDeviceToHost));
    if (status) CK(cudaMemcpy(status, c->ca.status, c->ncol, cudaMemcpyDeviceToHost));
    if (dmax) CK(cudaMemcpy(dmax, c->ca.dmax, c->ncol * 8, cudaMemcpyDeviceToHost));
    return RH_OK;
}

int rh_get_lte(rh_ctx *c, double *nstar_out, double *ne_out)
{
    if (!c) return RH_EINVAL;
    if (!c->ncol) return fail(c, RH_ESTATE, "no columns loaded");
    cudaSetDevice(c->dev);
    CK(cudaStreamSynchronize(c->st));
    size_t nd = (size_t)c->ncol * c->ndep;
    if (nstar_out) CK(cudaMemcpy(nstar_out, c->ca.nstar, nd * c->da.nlev * 8, cudaMemcpyDeviceToHost));
    if (ne_out) CK(cudaMemcpy(ne_out, c->ca.ne, nd * 8, cudaMemcpyDeviceToHost));
    return RH_OK;
}

int rh_column_smem_layout(int32_t precision, int32_t nlev, int32_t ndep, int32_t ntr, int32_t ncont, int32_t nline,
                          int32_t macc, int32_t ring_warps, size_t *offsets_out, size_t *bytes_out)
{
    if ((precision != 0 && precision != 1) || nlev < 2 || nlev > RH_MAXLEV || ndep < 2 || ndep > 4096 || ntr < 1 ||
        ntr > RH_MAXTR || ncont < 0 || nline < 0 || macc < 1 || ring_warps < 0 || ring_warps > 32 || !offsets_out ||
        !bytes_out)
        return RH_EINVAL;
    mali_smem_layout(precision, nlev, ndep, ntr, ncont, nline, macc, ring_warps, offsets_out, 16, bytes_out);
    return RH_OK;
}

int rh_get_columns(rh_ctx *c, double *z_out, double *T_out, double *nH_out, double *vz_out)
{
    if (!c) return RH_EINVAL;
    if (!c->ncol) return fail(c, RH_ESTATE, "no columns loaded");
    cudaSetDevice(c->dev);
    CK(cudaStreamSynchronize(c->st));
    const size_t nd = (size_t)c->ncol * c->ndep * 8;
    if (z_out) CK(cudaMemcpy(z_out, c->ca.z, nd, cudaMemcpyDeviceToHost));
    if (T_out) CK(cudaMemcpy(T_out, c->ca.T, nd, cudaMemcpyDeviceToHost));
    if (nH_out) CK(cudaMemcpy(nH_out, c->ca.nH, nd, cudaMemcpyDeviceToHost));
    if (vz_out) CK(cudaMemcpy(vz_out, c->ca.vz, nd, cudaMemcpyDeviceToHost));
    return RH_OK;
}

int rh_regrid(rh_ctx *c, int32_t ndep_out, const rh_grid_opts *o)
{
    if (!c) return RH_EINVAL;
    if (!c->ncol) return fail(c, RH_ESTATE, "rh_regrid: no columns loaded");
    if (!o || ndep_out < 2 || ndep_out > 4096 || !(o->dlog_colden > 0) || !(o->dlnT > 0) || !(o->dvz > 0) ||
        !(o->spacing_factor >= 1.0) || !std::isfinite(o->spacing_factor) || (o->use_z_top && !std::isfinite(o->z_top)))
        return fail(c, RH_EINVAL, "rh_regrid: invalid options");
    cudaSetDevice(c->dev);
    const int64_t nc = c->ncol;
    const size_t nout = (size_t)nc * ndep_out * 8;
    double *buf = nullptr, *srow = nullptr;
    unsigned long long *bad = nullptr;
    CK(cudaMalloc(&buf, 5 * nout));
    cudaError_t e = cudaMalloc(&srow, (size_t)nc * c->ndep * 8);
    if (e == cudaSuccess) e = cudaMalloc(&bad, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFree(buf);
        cudaFree(srow);
        return fail(c, RH_ENOMEM, "rh_regrid: %s", cudaGetErrorString(e));
    }
    double *zo = buf, *To = zo + nout / 8, *nHo = To + nout / 8, *vzo = nHo + nout / 8, *neo = vzo + nout / 8;
    RegridParams g{o->dlog_colden, o->dlnT, o->dvz, o->spacing_factor, o->z_top, o->use_z_top ? 1 : 0};
    unsigned long long hbad = ~0ull;
    e = cudaMemcpyAsync(bad, &hbad, sizeof hbad, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = launch_regrid(c->ca, ndep_out, g, srow, zo, To, nHo, vzo, neo, bad, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    int r = RH_OK;
    if (e != cudaSuccess) {
        r = fail(c, RH_ECUDA, "rh_regrid: %s", cudaGetErrorString(e));
    } else if (hbad != ~0ull) {
        r = fail(c, RH_EINVAL, "rh_regrid: z_top leaves no layer in column %llu", hbad);
    } else {
        // the new columns replace the old ones (copied; LTE set-up on the new grid)
        r = rh_load_columns(c, nc, ndep_out, zo, To, neo, nHo, vzo, 1);
    }
    cudaFree(buf);
    cudaFree(srow);
    cudaFree(bad);
    return r;
}

int rh_set_populations(rh_ctx *c, const double *n_in)
{
    if (!c || !n_in) return RH_EINVAL;
    if (!c->ncol) return fail(c, RH_ESTATE, "no columns loaded");
    size_t nv = (size_t)c->ncol * c->ndep * c->da.nlev;
    for (size_t i = 0; i < nv; ++i)
        if (!(std::isfinite(n_in[i]) && n_in[i] > 0))
            return fail(c, RH_EINVAL, "populations must be finite and > 0 (first bad flat index %zu)", i);
    cudaSetDevice(c->dev);
    CK(cudaMemcpy(c->ca.pops, n_in, nv * 8, cudaMemcpyHostToDevice));
    return RH_OK;
}

int rh_emergent_spectrum(rh_ctx *c, double mu, int64_t nlambda, const double *lambda_m, double *I_out,
                         int32_t precision, int32_t on_device)
{
    if (!c) return RH_EINVAL;
    if (!c->ncol) return fail(c, RH_ESTATE, "no columns loaded");
    if (!(mu > 0 && mu <= 1)) return fail(c, RH_EINVAL, "mu must be in (0, 1]");
    if (nlambda < 1 || !lambda_m || !I_out) return fail(c, RH_EINVAL, "need nlambda >= 1 and buffers");
    if (precision != 0 && precision != 1) return fail(c, RH_EINVAL, "precision must be 0 or 1");
    cudaSetDevice(c->dev);
    std::vector<double> nu, spec;
    std::vector<int> nact, act;
    int r0 = spectrum_tables(c, nlambda, lambda_m, nu, nact, act, spec);
    if (r0) return r0;
    double *nu_d = nullptr, *spec_d = nullptr, *out_d = nullptr;
    int *nact_d = nullptr, *act_d = nullptr;
    int rc = RH_OK;
    auto cleanup = [&]() {
        dfree(nu_d);
        dfree(spec_d);
        dfree(nact_d);
        dfree(act_d);
        if (!on_device) dfree(out_d);
    };
    cudaError_t e = cudaMalloc(&nu_d, nlambda * 8);
    if (e == cudaSuccess) e = cudaMalloc(&spec_d, spec.size() * 8);
    if (e == cudaSuccess) e = cudaMalloc(&nact_d, nlambda * 4);
    if (e == cudaSuccess) e = cudaMalloc(&act_d, act.size() * 4);
    if (e == cudaSuccess) {
        if (on_device) out_d = I_out;
        else e = cudaMalloc(&out_d, (size_t)c->ncol * nlambda * 8);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(nu_d, nu.data(), nlambda * 8, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(spec_d, spec.data(), spec.size() * 8, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nact_d, nact.data(), nlambda * 4, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(act_d, act.data(), act.size() * 4, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = launch_spectrum(c->da, c->ca, mu, nlambda, nu_d, nact_d, act_d, spec_d, out_d, precision, c->st);
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(I_out, out_d, (size_t)c->ncol * nlambda * 8, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) rc = fail(c, RH_ECUDA, "rh_emergent_spectrum: %s", cudaGetErrorString(e));
    cleanup();
    return rc;
}

int rh_emergent_stokes(rh_ctx *c, int32_t line, double g_eff, const double *B_T, const double *theta,
                       const double *chi, int64_t nlambda, const double *lambda_m, double *iquv_out,
                       int32_t precision, int32_t on_device)
{
    if (!c) return RH_EINVAL;
    if (!c->ncol) return fail(c, RH_ESTATE, "no columns loaded");
    if (line < 0 || line >= c->da.nline) return fail(c, RH_EINVAL, "rh_emergent_stokes: line index out of range");
    if (!std::isfinite(g_eff)) return fail(c, RH_EINVAL, "rh_emergent_stokes: g_eff must be finite");
    if (nlambda < 1 || !lambda_m || !iquv_out || !B_T || !theta || !chi)
        return fail(c, RH_EINVAL, "need nlambda >= 1 and buffers");
    if (precision != 0 && precision != 1) return fail(c, RH_EINVAL, "precision must be 0 or 1");
    if (on_device != 0 && on_device != 1) return fail(c, RH_EINVAL, "on_device must be 0 or 1");
    cudaSetDevice(c->dev);
    const size_t nd = (size_t)c->ncol * c->ndep;
    if (!on_device)
        for (size_t i = 0; i < nd; ++i)
            if (!std::isfinite(B_T[i]) || B_T[i] < 0 || !std::isfinite(theta[i]) || !std::isfinite(chi[i]))
                return fail(c, RH_EINVAL, "rh_emergent_stokes: field entry %zu not finite (or B < 0)", i);
    std::vector<double> nu, spec;
    std::vector<int> nact, act;
    int r0 = spectrum_tables(c, nlambda, lambda_m, nu, nact, act, spec);
    if (r0) return r0;
    double *nu_d = nullptr, *spec_d = nullptr, *out_d = nullptr, *fld = nullptr;
    int *nact_d = nullptr, *act_d = nullptr;
    auto cleanup = [&]() {
        dfree(nu_d);
        dfree(spec_d);
        dfree(nact_d);
        dfree(act_d);
        dfree(fld);
        if (!on_device) dfree(out_d);
    };
    const double *Bd = B_T, *td = theta, *cd = chi;
    cudaError_t e = cudaMalloc(&nu_d, nlambda * 8);
    if (e == cudaSuccess) e = cudaMalloc(&spec_d, spec.size() * 8);
    if (e == cudaSuccess) e = cudaMalloc(&nact_d, nlambda * 4);
    if (e == cudaSuccess) e = cudaMalloc(&act_d, act.size() * 4);
    if (e == cudaSuccess && !on_device) {
        e = cudaMalloc(&fld, 3 * nd * 8);
        if (e == cudaSuccess) e = cudaMemcpyAsync(fld, B_T, nd * 8, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(fld + nd, theta, nd * 8, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(fld + 2 * nd, chi, nd * 8, cudaMemcpyHostToDevice, c->st);
        Bd = fld;
        td = fld + nd;
        cd = fld + 2 * nd;
    }
    if (e == cudaSuccess) {
        if (on_device) out_d = iquv_out;
        else e = cudaMalloc(&out_d, (size_t)c->ncol * nlambda * 4 * 8);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(nu_d, nu.data(), nlambda * 8, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(spec_d, spec.data(), spec.size() * 8, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nact_d, nact.data(), nlambda * 4, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(act_d, act.data(), act.size() * 4, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess)
        e = launch_stokes(c->da, c->ca, line, g_eff, Bd, td, cd, nlambda, nu_d, nact_d, act_d, spec_d, c->vtab_d,
                          c->dtab_d, out_d, precision, c->st);
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(iquv_out, out_d, (size_t)c->ncol * nlambda * 4 * 8, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    int rc = RH_OK;
    if (e != cudaSuccess) rc = fail(c, RH_ECUDA, "rh_emergent_stokes: %s", cudaGetErrorString(e));
    cleanup();
    return rc;
}

}  // extern "C"

// ============================================================================
// rh_solve: pass 1 and the re-run passes of Sect. 2.3 with the selection of
// unconverged columns on the device, enqueued directly or captured once
// into a CUDA graph and replayed; rh_autotune: the launch shape of the
// column kernel.
namespace {

// Compact the indices of the columns whose status is not CONVERGED into
// colidx; count receives their number (warp-aggregated atomics: the order of
// colidx is not deterministic, the per-column results do not depend on it).
__global__ void select_unconverged_kernel(int64_t ncol, const uint8_t *status, int *colidx, int *count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool sel = i < ncol && status[i] != RH_COL_CONVERGED;
    const unsigned m = __ballot_sync(0xffffffffu, sel);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (sel) colidx[base + __popc(m & ((1u << lane) - 1u))] = (int)i;
}

// Sum of iters over the first n (or *count_d) work items into *out.
__global__ void sum_iters_kernel(int64_t n, const int *colidx, const int *count_d, const int32_t *iters,
                                 unsigned long long *out)
{
    const int64_t cnt = count_d ? (int64_t)*count_d : n;
    unsigned long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        s += (unsigned long long)iters[colidx ? colidx[i] : i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

bool valid_iter_opts(const rh_iter_opts *o)
{
    return o->maxiter >= 1 && o->tol >= 0 && (o->ng_order == 0 || o->ng_order == 2) &&
           !(o->ng_order == 2 && (o->ng_period < 1 || o->ng_delay < 0)) && (o->precision == 0 || o->precision == 1) &&
           o->start >= 0 && o->start <= 4 && o->block_warps >= 0 && o->block_warps <= 8 &&
           std::isfinite(o->prd_eps0) && (o->prd_hybrid == 0 || o->prd_hybrid == 1) &&
           (o->formal == 0 || o->formal == 1);
}

// everything the enqueued sequence depends on, compared byte-wise
struct SolveKey {
    const void *ptrs[31];
    int64_t ncol;
    int ndep, bw, ctas, nsm;
    rh_solve_opts o;
};

SolveKey make_key(const rh_ctx *c, const rh_solve_opts *o, int bw, int ctas)
{
    SolveKey k;
    memset(&k, 0, sizeof k);
    const void *p[] = {c->ca.z, c->ca.T, c->ca.nH, c->ca.vz, c->ca.ne, c->ca.np, c->ca.nstar, c->ca.pops,
                       c->ca.Crate, c->ca.dmax, c->ca.iters, c->ca.status, c->lane_d, c->vtab_d, c->nghist,
                       c->queue, c->colidx, c->solve_cnt, c->solve_it, c->mlp, c->feat, c->lnb, c->nfb_d, c->st,
                       c->sp_off_d, c->sp_nu_d, c->sp_ce_d, c->lane_prd_d, c->prd_nu_d, c->prd_w_d,
                       c->prd_scr};
    static_assert(sizeof p / sizeof p[0] == 31, "key size");
    memcpy(k.ptrs, p, sizeof p);
    k.ncol = c->ncol;
    k.ndep = c->ndep;
    k.bw = bw;
    k.ctas = ctas;
    k.nsm = c->nsm;
    memcpy(&k.o, o, sizeof *o);
    k.o.pass1.only_unconverged = 0;
    return k;
}

// Enqueue the whole sequence on c->st; counts the kernels it launches.
// end-of-pass timing events: external event nodes when the sequence is captured
cudaError_t record_pass_end(rh_ctx *c, int i, bool capturing)
{
    return capturing ? cudaEventRecordWithFlags(c->pass_ev[i], c->st, cudaEventRecordExternal)
                     : cudaEventRecord(c->pass_ev[i], c->st);
}

cudaError_t enqueue_solve(rh_ctx *c, const rh_solve_opts *o, const IterLaunch &base, char *err, size_t errn,
                          int *nkern, bool capturing)
{
    cudaStream_t st = c->st;
    int nk = 0;
    cudaError_t e = cudaMemsetAsync(c->solve_cnt, 0, RH_MAX_RERUN * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->solve_it, 0, (1 + RH_MAX_RERUN) * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (o->pass1.start == 1) {
        if ((e = mlp_predict_apply(c->mlp, c->ca, c->da.nlev, c->feat, c->lnb, c->nfb_d, st)) != cudaSuccess) return e;
        const int64_t nchunk = (c->ncol + 16383) / 16384;
        nk += 2 + (int)nchunk * (1 + mlp_nlayer(c->mlp));
    } else if (o->pass1.start == 3 || o->pass1.start == 4) {
        if ((e = launch_start(c->da, c->ca, o->pass1.start, c->sp_off_d, c->sp_nu_d, c->sp_ce_d, st)) != cudaSuccess)
            return e;
        nk += 1;
    }
    const int sgrid = 2 * c->nsm;
    IterLaunch il = base;
    il.start = o->pass1.start == 0 ? 0 : 2;
    il.colidx = nullptr;
    il.nwork = c->ncol;
    il.nwork_d = nullptr;
    int grid = 0;
    if (o->fused_rerun) {
        // one launch: the kernel re-runs failing columns itself and counts
        il.nrung = o->nrerun;
        il.rung_maxiter = o->rerun_maxiter;
        for (int r = 0; r < o->nrerun; ++r) {
            il.rung_crsw[r] = o->rerun_crsw[r];
            il.rung_ng[r] = o->rerun_ng[r] ? o->pass1.ng_order : 0;
        }
        il.rung_cols = c->solve_cnt;
        il.rung_its = c->solve_it;
        if ((e = launch_mali_prealloc(c->da, c->ca, c->lane_d, c->ha.npad, c->vtab_d, c->nref, c->nghist,
                                      c->nghist_cap, c->queue, il, st, &grid, err, errn)) != cudaSuccess)
            return e;
        *nkern = nk + 1;
        if ((e = record_pass_end(c, 0, capturing)) != cudaSuccess) return e;
        for (int r = 0; r < o->nrerun; ++r)
            if ((e = record_pass_end(c, 1 + r, capturing)) != cudaSuccess) return e;
        return cudaGetLastError();
    }
    if ((e = launch_mali_prealloc(c->da, c->ca, c->lane_d, c->ha.npad, c->vtab_d, c->nref, c->nghist, c->nghist_cap,
                                  c->queue, il, st, &grid, err, errn)) != cudaSuccess)
        return e;
    sum_iters_kernel<<<sgrid, 256, 0, st>>>(c->ncol, nullptr, nullptr, c->ca.iters, c->solve_it);
    nk += 2;
    if ((e = record_pass_end(c, 0, capturing)) != cudaSuccess) return e;
    for (int r = 0; r < o->nrerun; ++r) {
        select_unconverged_kernel<<<(unsigned)((c->ncol + 255) / 256), 256, 0, st>>>(c->ncol, c->ca.status, c->colidx,
                                                                                   c->solve_cnt + r);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        IterLaunch ir = base;
        ir.start = 0;
        ir.ng_order = o->rerun_ng[r] ? o->pass1.ng_order : 0;
        ir.crsw = o->rerun_crsw[r];
        ir.maxiter = o->rerun_maxiter;
        ir.colidx = c->colidx;
        ir.nwork = c->ncol;
        ir.nwork_d = c->solve_cnt + r;
        if ((e = launch_mali_prealloc(c->da, c->ca, c->lane_d, c->ha.npad, c->vtab_d, c->nref, c->nghist,
                                      c->nghist_cap, c->queue, ir, st, &grid, err, errn)) != cudaSuccess)
            return e;
        sum_iters_kernel<<<sgrid, 256, 0, st>>>(c->ncol, c->colidx, c->solve_cnt + r, c->ca.iters, c->solve_it + 1 + r);
        nk += 3;
        if ((e = record_pass_end(c, 1 + r, capturing)) != cudaSuccess) return e;
    }
    *nkern = nk;
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int rh_start_populations(rh_ctx *c, int32_t kind)
{
    if (!c) return RH_EINVAL;
    if (!c->ncol) return fail(c, RH_ESTATE, "rh_start_populations: no columns loaded");
    if (kind != 0 && kind != 1 && kind != 3 && kind != 4)
        return fail(c, RH_EINVAL, "rh_start_populations: kind 0, 1, 3 or 4");
    cudaSetDevice(c->dev);
    const size_t nv = (size_t)c->ncol * c->ndep * c->da.nlev;
    if (kind == 0) {
        CK(cudaMemcpyAsync(c->ca.pops, c->ca.nstar, nv * 8, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemsetAsync(c->ca.status, RH_COL_NOTRUN, c->ncol, c->st));
    } else if (kind == 1) {
        if (!c->mlp || c->mlp_ndep != c->ndep)
            return fail(c, RH_ESTATE, "rh_start_populations: kind 1 needs a surrogate for %d depths", c->ndep);
        drop_graph(c);   // network buffers may be (re)allocated
        int r = ensure_mlp_buffers(c);
        if (r) return r;
        CK(mlp_predict_apply(c->mlp, c->ca, c->da.nlev, c->feat, c->lnb, c->nfb_d, c->st));
        CK(cudaMemsetAsync(c->ca.status, RH_COL_NOTRUN, c->ncol, c->st));
    } else {
        int r = ensure_start_tables(c);
        if (r) return r;
        CK(launch_start(c->da, c->ca, kind, c->sp_off_d, c->sp_nu_d, c->sp_ce_d, c->st));
    }
    CK(cudaStreamSynchronize(c->st));
    return RH_OK;
}

int rh_autotune(rh_ctx *c, int32_t precision, rh_tune_result *out)
{
    if (!c) return RH_EINVAL;
    if (!c->ncol) return fail(c, RH_ESTATE, "rh_autotune: no columns loaded");
    if (precision != 0 && precision != 1) return fail(c, RH_EINVAL, "rh_autotune: precision 0 or 1");
    cudaSetDevice(c->dev);
    int r = ensure_lane(c, precision);
    if (r) return r;
    r = ensure_prd(c, precision);
    if (r) return r;
    r = ensure_phic(c, precision);
    if (r) return r;
    const size_t per_block = mali_nghist_bytes_per_block(c->da, c->ndep);
    const size_t want = per_block * (size_t)c->nsm * 4;
    if (c->nghist_cap < want) {
        drop_graph(c);
        dfree(c->nghist);
        c->nghist_cap = 0;
        CK(cudaMalloc(&c->nghist, want));
        c->nghist_cap = want;
    }
    const int L = c->da.nlev, N = c->ndep;
    const int64_t S = std::min<int64_t>(c->ncol, (int64_t)4 * c->nsm);
    // keep the sample columns' state: the candidates overwrite it
    double *sv_n = nullptr, *sv_d = nullptr;
    int32_t *sv_i = nullptr;
    uint8_t *sv_s = nullptr;
    CK(cudaMalloc(&sv_n, (size_t)S * L * N * 8));
    CK(cudaMalloc(&sv_d, S * 8));
    CK(cudaMalloc(&sv_i, S * 4));
    CK(cudaMalloc(&sv_s, S));
    auto cleanup = [&]() {
        cudaFree(sv_n);
        cudaFree(sv_d);
        cudaFree(sv_i);
        cudaFree(sv_s);
    };
    cudaError_t e = cudaMemcpyAsync(sv_n, c->ca.pops, (size_t)S * L * N * 8, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sv_d, c->ca.dmax, S * 8, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sv_i, c->ca.iters, S * 4, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sv_s, c->ca.status, S, cudaMemcpyDeviceToDevice, c->st);
    rh_tune_result R;
    memset(&R, 0, sizeof R);
    R.sample_columns = S;
    // warps per column block: a block's warps share the 32-wavelength tiles of
    // its column, so counts that divide the tile count into nearly whole
    // rounds (19 tiles: 7 warps fill 19 of 21 warp-slots, 8 warps 19 of 24)
    // leave fewer warps idle at the end of the sweep
    const int bws[4] = {precision ? 4 : 2, precision ? 6 : 4, precision ? 7 : 8, 8};
    const int nbw = precision ? 4 : 3;
    for (int ib = 0; ib < nbw && e == cudaSuccess; ++ib) {
        const int maxc = mali_max_ctas_per_sm(c->da, N, precision, bws[ib]);
        for (int ct = 1; ct <= std::min(maxc, 2) && R.ncand < RH_MAX_TUNE; ++ct) {
            IterLaunch il;
            il.precision = precision;
            il.persistent = 1;
            il.block_warps = bws[ib];
            il.ctas_per_sm = ct;
            il.maxiter = 2;
            il.tol = 0.0;
            il.start = 0;
            il.nsm = c->nsm;
            il.nwork = S;
            set_prd(c, il, 0.0, 0);
            set_phic(c, il);
            double best = -1;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // first run: warm-up
                float ms = 0;
                int grid = 0;
                char eb[256] = {0};
                e = launch_mali(c->da, c->ca, c->lane_d, c->ha.npad, c->vtab_d, c->nref, c->nghist, c->nghist_cap,
                                c->queue, il, c->st, &ms, &grid, eb, sizeof eb);
                if (rep == 1) best = ms;
            }
            R.cand_block_warps[R.ncand] = bws[ib];
            R.cand_ctas_per_sm[R.ncand] = ct;
            R.cand_ms[R.ncand] = best;
            R.ncand++;
        }
        if (maxc < 1 && R.ncand < RH_MAX_TUNE) {
            R.cand_block_warps[R.ncand] = bws[ib];
            R.cand_ctas_per_sm[R.ncand] = 0;
            R.cand_ms[R.ncand] = -1;
            R.ncand++;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ca.pops, sv_n, (size_t)S * L * N * 8, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ca.dmax, sv_d, S * 8, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ca.iters, sv_i, S * 4, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ca.status, sv_s, S, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    cleanup();
    if (e != cudaSuccess) return fail(c, RH_ECUDA, "rh_autotune: %s", cudaGetErrorString(e));
    int bi = -1;
    for (int i = 0; i < R.ncand; ++i)
        if (R.cand_ms[i] > 0 && (bi < 0 || R.cand_ms[i] < R.cand_ms[bi])) bi = i;
    if (bi < 0) return fail(c, RH_ECUDA, "rh_autotune: no launch shape fits");
    R.best_block_warps = R.cand_block_warps[bi];
    R.best_ctas_per_sm = R.cand_ctas_per_sm[bi];
    c->tuned_bw[precision] = R.best_block_warps;
    c->tuned_ctas[precision] = R.best_ctas_per_sm;
    drop_graph(c);
    if (out) *out = R;
    return RH_OK;
}

int rh_solve(rh_ctx *c, const rh_solve_opts *o, rh_solve_stats *st)
{
    if (!c) return RH_EINVAL;
    if (!c->ncol) return fail(c, RH_ESTATE, "rh_solve: no columns loaded");
    if (!o) return fail(c, RH_EINVAL, "opts is NULL");
    if (!valid_iter_opts(&o->pass1) || o->nrerun < 0 || o->nrerun > RH_MAX_RERUN ||
        (o->nrerun > 0 && o->rerun_maxiter < 1) || (o->use_graph != 0 && o->use_graph != 1) ||
        (o->autotune != 0 && o->autotune != 1) || (o->fused_rerun != 0 && o->fused_rerun != 1))
        return fail(c, RH_EINVAL, "rh_solve: invalid options");
    for (int r = 0; r < o->nrerun; ++r)
        if (!(o->rerun_crsw[r] >= 1.0) || (o->rerun_ng[r] != 0 && o->rerun_ng[r] != 1))
            return fail(c, RH_EINVAL, "rh_solve: rerun_crsw must be >= 1 and rerun_ng 0 or 1");
    cudaSetDevice(c->dev);
    const int prec = o->pass1.precision;
    if (o->pass1.start == 1) {
        if (!c->mlp || c->mlp_ndep != c->ndep)
            return fail(c, RH_ESTATE, "rh_solve: start = 1 needs a surrogate for %d depths (rh_surrogate_init)",
                        c->ndep);
        int r = ensure_mlp_buffers(c);
        if (r) return r;
        CK(mlp_prepare_predict(c->mlp, c->ncol));
    }
    if (o->pass1.start == 3 || o->pass1.start == 4) {
        int r = ensure_start_tables(c);
        if (r) return r;
    }
    if (o->autotune && o->pass1.block_warps == 0 && !c->tuned_bw[prec]) {
        int r = rh_autotune(c, prec, nullptr);
        if (r) return r;
    }
    // everything the sequence touches exists before it is enqueued or captured
    int r = ensure_lane(c, prec);
    if (r) return r;
    r = ensure_prd(c, prec);
    if (r) return r;
    r = ensure_phic(c, prec);
    if (r) return r;
    const size_t per_block = mali_nghist_bytes_per_block(c->da, c->ndep);
    const size_t want = per_block * (size_t)c->nsm * 4;
    if (c->nghist_cap < want) {
        dfree(c->nghist);
        c->nghist_cap = 0;
        CK(cudaMalloc(&c->nghist, want));
        c->nghist_cap = want;
    }
    if (c->colidx_cap < c->ncol) {
        dfree(c->colidx);
        CK(cudaMalloc(&c->colidx, c->ncol * sizeof(int)));
        c->colidx_cap = c->ncol;
    }
    for (cudaEvent_t &ev : c->pass_ev)
        if (!ev) CK(cudaEventCreate(&ev));
    if (!c->solve_cnt) CK(cudaMalloc(&c->solve_cnt, RH_MAX_RERUN * sizeof(int)));
    if (!c->solve_it) CK(cudaMalloc(&c->solve_it, (1 + RH_MAX_RERUN) * sizeof(unsigned long long)));

    IterLaunch base;
    base.precision = prec;
    base.formal = o->pass1.formal;
    base.persistent = o->pass1.persistent;
    base.block_warps = o->pass1.block_warps;
    base.maxiter = o->pass1.maxiter;
    base.ng_order = o->pass1.ng_order;
    base.ng_delay = o->pass1.ng_delay;
    base.ng_period = o->pass1.ng_period;
    base.tol = o->pass1.tol;
    base.crsw = o->pass1.crsw_init;
    base.nsm = c->nsm;
    if (o->pass1.block_warps == 0 && c->tuned_bw[prec]) {
        base.block_warps = c->tuned_bw[prec];
        base.ctas_per_sm = c->tuned_ctas[prec];
    }
    set_prd(c, base, o->pass1.prd_eps0, o->pass1.prd_hybrid);
    set_phic(c, base);
    const int bw_used = base.block_warps > 0 ? base.block_warps : (prec ? 8 : 4);
    const int ctas_max = mali_max_ctas_per_sm(c->da, c->ndep, prec, bw_used);
    const int ctas_used = base.ctas_per_sm > 0 ? std::min(base.ctas_per_sm, ctas_max) : ctas_max;

    char eb[256] = {0};
    int replayed = 0, nkern = 0;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    cudaError_t e = cudaSuccess;
    if (o->use_graph) {
        SolveKey k = make_key(c, o, bw_used, ctas_used);
        const unsigned char *kb = reinterpret_cast<const unsigned char *>(&k);
        if (!(c->gexec && c->gkey.size() == sizeof k && memcmp(c->gkey.data(), kb, sizeof k) == 0)) {
            drop_graph(c);
            e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t eq = enqueue_solve(c, o, base, eb, sizeof eb, &nkern, true);
                cudaGraph_t g = nullptr;
                e = cudaStreamEndCapture(c->st, &g);
                if (eq != cudaSuccess) e = eq;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, g, 0);
                if (e == cudaSuccess) {
                    c->graph = g;
                    c->gkey.assign(kb, kb + sizeof k);
                    c->glaunches = nkern;
                } else if (g) {
                    cudaGraphDestroy(g);
                }
            }
        } else {
            replayed = 1;
        }
        nkern = c->glaunches;
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->st);
        if (e == cudaSuccess) e = cudaGraphLaunch(c->gexec, c->st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->st);
    } else {
        e = cudaEventRecord(e0, c->st);
        if (e == cudaSuccess) e = enqueue_solve(c, o, base, eb, sizeof eb, &nkern, false);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->st);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0, pms[1 + RH_MAX_RERUN] = {};
    if (e == cudaSuccess) {
        cudaEventElapsedTime(&ms, e0, e1);
        for (int i = 0; i <= o->nrerun; ++i) cudaEventElapsedTime(&pms[i], i ? c->pass_ev[i - 1] : e0, c->pass_ev[i]);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        drop_graph(c);
        return fail(c, RH_ECUDA, "rh_solve: %s%s%s", cudaGetErrorString(e), eb[0] ? ": " : "", eb);
    }
    int cnt[RH_MAX_RERUN];
    unsigned long long its[1 + RH_MAX_RERUN];
    int nfb = 0;
    CK(cudaMemcpy(cnt, c->solve_cnt, sizeof cnt, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(its, c->solve_it, sizeof its, cudaMemcpyDeviceToHost));
    if (o->pass1.start == 1) CK(cudaMemcpy(&nfb, c->nfb_d, sizeof nfb, cudaMemcpyDeviceToHost));
    std::vector<uint8_t> s(c->ncol);
    CK(cudaMemcpy(s.data(), c->ca.status, c->ncol, cudaMemcpyDeviceToHost));
    rh_solve_stats S;
    memset(&S, 0, sizeof S);
    for (int64_t i = 0; i < c->ncol; ++i) {
        if (s[i] == RH_COL_CONVERGED) S.n_converged++;
        else if (s[i] == RH_COL_MAXITER) S.n_maxiter++;
        else S.n_failed++;
    }
    S.pass_columns[0] = c->ncol;
    S.pass_iterations[0] = (int64_t)its[0];
    S.iterations_total = (int64_t)its[0];
    for (int r2 = 0; r2 < o->nrerun; ++r2) {
        S.pass_columns[1 + r2] = cnt[r2];
        S.pass_iterations[1 + r2] = (int64_t)its[1 + r2];
        S.iterations_total += (int64_t)its[1 + r2];
    }
    S.seconds = ms * 1e-3;
    for (int i = 0; i <= o->nrerun; ++i) S.pass_seconds[i] = pms[i] * 1e-3;
    S.pts = (double)S.iterations_total * c->ndep * (double)c->ha.nu.size() * c->ha.nmu;
    S.guess_fallback_depths = nfb;
    S.kernel_launches = nkern;
    S.graph_replayed = replayed;
    S.block_warps = bw_used;
    S.ctas_per_sm = ctas_used;
    if (st) *st = S;
    return (S.n_maxiter || S.n_failed) ? RH_ENOTCONV : RH_OK;
}

}  // extern "C"

// ============================================================================
// rh_iterate_noalloc: the MALI iteration for callers that cannot allocate
// device memory at solve time (see include/rh15d.h).  Its scratch -- the
// work-queue counter, result counters, the lane table in the iteration's
// precision, and the Ng history of the resident blocks -- lives in one
// file-scope device array that every GPU loading this library holds until
// the process exits.
namespace {

constexpr size_t kNoallocBytes = (size_t)9 << 20;              // 9 MiB in total
constexpr size_t kNoallocHead = 256;                           // queue counter + 4 result counters
constexpr size_t kNoallocLaneBytes = (size_t)kLaneFields * RH_MAXTILE * 32 * sizeof(double);
constexpr size_t kNoallocHistOff = kNoallocHead + ((kNoallocLaneBytes + 255) / 256) * 256;
constexpr size_t kNoallocHistBytes = kNoallocBytes - kNoallocHistOff;
constexpr int kNoallocMaxDev = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// device address of the scratch array, looked up once per device (host code
// may not use the symbol itself as an address)
void *g_noalloc_dev_ptr[kNoallocMaxDev];
// host staging of the lane table (static: no heap allocation per call),
// shared by every call; the lock serialises calls from several host threads
// while they fill it and hand it to cudaMemcpyAsync (which has copied a
// pageable source out by the time it returns)
double g_noalloc_lane64[(size_t)kLaneFields * RH_MAXTILE * 32];
float g_noalloc_lane32[(size_t)kLaneFields * RH_MAXTILE * 32];
std::mutex g_noalloc_mutex;

// restores the caller's current device when the call returns
struct DeviceRestore {
    int dev = -1;
    DeviceRestore() { if (cudaGetDevice(&dev) != cudaSuccess) dev = -1; }
    ~DeviceRestore() { if (dev >= 0) cudaSetDevice(dev); }
};

// 1 if p is device (or managed) memory of device dev
bool noalloc_device_pointer(const void *p, int dev)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // clear the sticky-free error of an unknown pointer
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

__global__ void noalloc_count_kernel(int64_t ncol, const int32_t *iters, const uint8_t *status,
                                     unsigned long long *cnt)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncol) return;
    const uint8_t s = status[i];
    atomicAdd(&cnt[s == RH_COL_CONVERGED ? 0 : (s == RH_COL_MAXITER ? 1 : 2)], 1ull);
    atomicAdd(&cnt[3], (unsigned long long)iters[i]);
}

// max over columns of dmax (NaN entries skipped, as in rh_iterate; the
// column kernel writes none); the kernel writes only values >= 0
__global__ void noalloc_max_kernel(int64_t ncol, const double *dmax, unsigned long long *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncol) return;
    const double v = dmax[i];
    if (v >= 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(v));   // non-negative doubles order as bits
}

}  // namespace

extern "C" int rh_iterate_noalloc(rh_ctx *c, const rh_iter_opts *o, double *n_out, int32_t *iters_out,
                                  uint8_t *status_out, double *dmax_out, rh_iter_stats *stats_out)
{
    if (!c) return RH_EINVAL;
    if (!c->ncol) return fail(c, RH_ESTATE, "rh_iterate_noalloc: no columns loaded");
    if (!o || !n_out || !iters_out || !status_out || !dmax_out)
        return fail(c, RH_EINVAL, "rh_iterate_noalloc: opts and the four output buffers must not be NULL");
    if (o->maxiter < 1 || !(o->tol >= 0) || (o->ng_order != 0 && o->ng_order != 2) ||
        (o->ng_order == 2 && (o->ng_period < 1 || o->ng_delay < 0)) || (o->precision != 0 && o->precision != 1) ||
        (o->start != 0 && o->start != 2) || o->block_warps < 0 || o->block_warps > 8 || o->only_unconverged != 0 ||
        (o->formal != 0 && o->formal != 1))
        return fail(c, RH_EINVAL, "rh_iterate_noalloc: invalid options (only_unconverged is not supported here)");
    if (c->da.nprd) return fail(c, RH_EINVAL, "rh_iterate_noalloc: atoms with PRD lines need scratch; use rh_iterate");
    if (c->dev < 0 || c->dev >= kNoallocMaxDev) return fail(c, RH_EINVAL, "rh_iterate_noalloc: device index too large");
    DeviceRestore restore_device;
    CK(cudaSetDevice(c->dev));
    {
        const void *bufs[4] = {n_out, iters_out, status_out, dmax_out};
        const char *names[4] = {"n_out", "iters_out", "status_out", "dmax_out"};
        for (int i = 0; i < 4; ++i)
            if (!noalloc_device_pointer(bufs[i], c->dev))
                return fail(c, RH_EINVAL, "rh_iterate_noalloc: %s is not device memory of device %d", names[i],
                            c->dev);
    }
    // once per device, with the device current: the scratch array's address
    if (!g_noalloc_dev_ptr[c->dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(c, RH_ECUDA, "rh_iterate_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_noalloc_dev_ptr[c->dev] = ptr;
    }
    unsigned char *base = (unsigned char *)g_noalloc_dev_ptr[c->dev];
    int *queue = (int *)base;
    unsigned long long *cnt = (unsigned long long *)(base + 64);
    void *lane = base + kNoallocHead;
    double *hist = (double *)(base + kNoallocHistOff);
    const size_t per_block = mali_nghist_bytes_per_block(c->da, c->ndep);
    if (per_block > kNoallocHistBytes)
        return fail(c, RH_EINVAL, "rh_iterate_noalloc: Ng history of one column needs %zu B, the scratch holds %zu B",
                    per_block, kNoallocHistBytes);
    // the lane table in the iteration's precision, populations scaled by n_ref
    const int np = c->ha.npad;
    const size_t nl = (size_t)kLaneFields * np;
    std::lock_guard<std::mutex> staging_lock(g_noalloc_mutex);
    for (size_t i = 0; i < nl; ++i) g_noalloc_lane64[i] = c->lane_master[i];
    for (int j = 0; j < RH_KMAX; ++j)
        for (int f : {1, 2})
            for (int p = 0; p < np; ++p) g_noalloc_lane64[(size_t)(RH_NLANEF * j + f) * np + p] *= c->nref;
    if (o->precision == 1) {
        for (size_t i = 0; i < nl; ++i) g_noalloc_lane32[i] = (float)g_noalloc_lane64[i];
        CK(cudaMemcpyAsync(lane, g_noalloc_lane32, nl * sizeof(float), cudaMemcpyHostToDevice, c->st));
    } else {
        CK(cudaMemcpyAsync(lane, g_noalloc_lane64, nl * sizeof(double), cudaMemcpyHostToDevice, c->st));
    }
    ColumnArrays cc = c->ca;
    cc.pops = n_out;
    cc.iters = iters_out;
    cc.status = status_out;
    cc.dmax = dmax_out;
    IterLaunch il{};
    il.precision = o->precision;
    il.formal = o->formal;
    il.persistent = o->persistent;
    il.block_warps = o->block_warps;
    il.maxiter = o->maxiter;
    il.ng_order = o->ng_order;
    il.ng_delay = o->ng_delay;
    il.ng_period = o->ng_period;
    il.start = o->start;
    il.tol = o->tol;
    il.crsw = o->crsw_init;
    il.nsm = c->nsm;
    il.colidx = nullptr;
    il.nwork = c->ncol;
    // the context's line-profile cache, when an earlier rh_iterate or rh_solve
    // allocated it (then this call runs the very kernel rh_iterate runs);
    // without it the sweep evaluates the profiles itself
    set_phic(c, il);
    int grid = 0;
    char ebuf[256] = {0};
    const std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    cudaError_t e = launch_mali_prealloc(c->da, cc, lane, np, c->vtab_d, c->nref, hist, kNoallocHistBytes, queue, il,
                                         c->st, &grid, ebuf, sizeof ebuf);
    if (e != cudaSuccess)
        return fail(c, RH_ECUDA, "rh_iterate_noalloc: %s%s%s", cudaGetErrorString(e), ebuf[0] ? ": " : "", ebuf);
    unsigned long long h[5] = {0, 0, 0, 0, 0};
    CK(cudaMemsetAsync(cnt, 0, 5 * sizeof(unsigned long long), c->st));
    noalloc_count_kernel<<<(unsigned)((c->ncol + 255) / 256), 256, 0, c->st>>>(c->ncol, iters_out, status_out, cnt);
    CK(cudaGetLastError());
    noalloc_max_kernel<<<(unsigned)((c->ncol + 255) / 256), 256, 0, c->st>>>(c->ncol, dmax_out, cnt + 4);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats_out) {
        rh_iter_stats S{};
        S.n_converged = (int64_t)h[0];
        S.n_maxiter = (int64_t)h[1];
        S.n_failed = (int64_t)h[2];
        S.n_processed = c->ncol;
        S.iterations_total = (int64_t)h[3];
        S.seconds = secs;
        S.pts = (double)S.iterations_total * c->ndep * (double)c->ha.nu.size() * c->ha.nmu;
        memcpy(&S.max_dn_final, &h[4], sizeof(double));
        *stats_out = S;
    }
    return (h[1] || h[2]) ? RH_ENOTCONV : RH_OK;
}
