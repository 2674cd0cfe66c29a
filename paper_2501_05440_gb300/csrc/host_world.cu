// host_world.cu -- flattening of problem definitions into device tables.
//
// Every array of every problem goes into one contiguous staging buffer (256-B
// aligned sub-arrays) and one device allocation; indices are made global with
// per-problem offsets so that a batch of problems is one World.  Derived
// per-group constants (mean free path, fission yield and its floor/fraction,
// scattering probability, cumulative distributions) are rounded once here.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "host_world.h"

namespace mcgb {

// The logarithm's tables, computed exactly enough in 128-bit fixed point with
// 120 fraction bits (Q120): a product of two Q120 numbers below 2^121 keeps
// its top bits from three 64-bit partial products (truncation below 3 units).
typedef unsigned __int128 u128;

static u128 mul_q120(u128 a, u128 b)
{
    const uint64_t ah = (uint64_t)(a >> 64), al = (uint64_t)a, bh = (uint64_t)(b >> 64),
                   bl = (uint64_t)b;
    const u128 hh = (u128)ah * bh, mid = (u128)ah * bl + (u128)al * bh, ll = (u128)al * bl;
    return (hh << 8) + (mid >> 56) + (ll >> 120);
}

// 2 atanh(num / den) = ln((den + num) / (den - num)) in Q120 for num/den <= 1/3:
// 2 (s + s^3/3 + s^5/5 + ...), summed until the terms vanish (error ~1e-33).
static u128 atanh2_q120(uint64_t num, uint64_t den)
{
    const u128 s = ((u128)num << 120) / den;
    const u128 z = mul_q120(s, s);
    u128 term = s, sum = 0;
    for (int k = 0; k < 256 && term; k++) {
        sum += term / (u128)(2 * k + 1);
        term = mul_q120(term, z);
    }
    return 2 * sum;
}

static int64_t q120_to_q57(u128 v) { return (int64_t)((v + ((u128)1 << 62)) >> 63); }

// ln(1 + j/256) in Q57, rounded to nearest: 2 atanh(j / (512 + j)).
int64_t ln_table_q57(int j) { return q120_to_q57(atanh2_q120((uint64_t)j, (uint64_t)(512 + j))); }

// ln 2 in Q57: 2 atanh(1/3).
int64_t ln2_q57() { return q120_to_q57(atanh2_q120(1, 3)); }

// Partial sums in order divided by the total; the last entry is exactly 1.
void make_cdf(const double *w, int n, double *cdf)
{
    double acc = 0.0;
    for (int k = 0; k < n; k++) {
        acc = acc + w[k];
        cdf[k] = acc;
    }
    for (int k = 0; k < n; k++) cdf[k] = cdf[k] / acc;
    cdf[n - 1] = 1.0;
}

std::string ProblemDef::check() const
{
    if (src.kind < 0) return "no source defined";
    if (cells.empty()) return "no cells defined";
    if (ce < 0) return "no materials defined";
    int nmat = ce ? (int)mce.size() : (int)mg.size();
    if (nmat == 0) return "no materials defined";
    int nu = 0;
    for (auto &c : cells) nu = std::max(nu, c.univ + 1);
    std::vector<int> ucount(nu, 0);
    for (auto &c : cells) ucount[c.univ]++;
    if (ucount[0] == 0) return "root universe 0 has no cells";
    int ns = (int)s_type.size();
    for (size_t i = 0; i < cells.size(); i++) {
        auto &c = cells[i];
        for (size_t h = 0; h < c.surf.size(); h++) {
            if (c.surf[h] < 0 || c.surf[h] >= ns) return "cell " + std::to_string(i) + ": bad surface";
            if (c.univ != 0 && s_bc[c.surf[h]] != BC_NONE)
                return "cell " + std::to_string(i) + ": boundary conditions apply to root cells only";
        }
        if (c.fillk == FILL_MAT && (c.fill < 0 || c.fill >= nmat))
            return "cell " + std::to_string(i) + ": bad material";
        if (c.fillk == FILL_LAT) {
            if (c.univ != 0) return "lattices may fill root cells only";
            if (c.fill < 0 || c.fill >= (int)lats.size()) return "cell " + std::to_string(i) + ": bad lattice";
        }
    }
    for (auto &L : lats)
        for (int u : L.univ) {
            if (u <= 0 || u >= nu || ucount[u] == 0) return "lattice refers to an empty universe";
        }
    for (auto &c : cells)
        if (c.univ != 0 && c.fillk != FILL_MAT) return "universe cells must hold materials";
    for (auto &t : tallies) {
        if (t.filter == FILTER_LATTICE && lats.empty()) return "lattice tally without a lattice";
        if (ce && t.edges.size() < 2) return "continuous-energy tally needs energy edges";
        if (!t.tedges.empty()) {
            if (t.tedges.size() < 2) return "time bins need at least two edges";
            for (size_t k = 0; k + 1 < t.tedges.size(); k++)
                if (!(t.tedges[k + 1] > t.tedges[k])) return "time edges must increase";
        }
    }
    if (time_on) {
        if (!(t0 >= 0.0) || !(tcut > t0) || !std::isfinite(tcut)) return "need 0 <= t0 < t_cut < inf";
        if (!ce) {
            if ((int)invv.size() != G) return "one inverse speed per group needed";
            for (double x : invv)
                if (!(x > 0.0) || !std::isfinite(x)) return "inverse speeds must be positive";
        }
    }
    if (!ce && src.ekind == E_PDF && (int)src.pdf.size() != G) return "source group pdf size != G";
    if (ce) {
        for (auto &m : mce)
            if ((int)m.nuc.size() > MAX_NUC) return "too many nuclides in a material";
    }
    return "";
}

DeviceWorld::~DeviceWorld()
{
    if (arena) cudaFree(arena);
}

namespace {

struct Staging {
    std::vector<char> buf;
    template <class T> size_t put(const std::vector<T> &v)
    {
        size_t off = (buf.size() + 255) & ~(size_t)255;
        buf.resize(off + std::max<size_t>(v.size() * sizeof(T), 8));
        if (!v.empty()) std::memcpy(buf.data() + off, v.data(), v.size() * sizeof(T));
        return off;
    }
};

}  // namespace

std::string build_world(const std::vector<ProblemRun> &runs, DeviceWorld &dw, cudaStream_t st)
{
    std::vector<int> s_type, s_bc;
    std::vector<double> s_coef, s_r2;
    std::vector<int> s_zc;
    std::vector<int> c_univ, c_off, c_nhs, c_fillk, c_fill, hs_surf, hs_sense;
    std::vector<double> l_x0, l_y0, l_pitch;
    std::vector<int> l_nx, l_ny, l_uoff, l_univ, l_woff;
    std::vector<double> l_wall, l_ctr;
    std::vector<int> m_G, m_goff, m_ggoff, m_fissile;
    std::vector<double> g_sigt, g_mfp, g_nusf, g_mu, g_mufl, g_mufr, g_ps, g_stot, g_chicdf;
    std::vector<double> gg_sigs, gg_scdf;
    std::vector<const NucDef *> nucs;
    std::vector<double> n_A, n_nu, n_kin;
    std::vector<int> mc_off, mc_n, mc_nuc, mc_fissile;
    std::vector<double> mc_dens, src_cdf;
    std::vector<int> t_filter, t_nbins, t_ne, t_off, t_eoff, t_nedges, t_batches, t_ntb, t_toff;
    std::vector<double> t_edges, t_tedges, t_tinvw, g_invv;
    std::vector<ProblemDev> probs;
    int nuniv = 0;
    int64_t acc_size = 0;
    std::vector<int> tally_first;

    for (const ProblemRun &r : runs) {
        const ProblemDef &pd = *r.def;
        std::string err = pd.check();
        if (!err.empty()) return err;
        ProblemDev P;
        std::memset(&P, 0, sizeof P);
        int surf0 = (int)s_type.size(), univ0 = nuniv, lat0 = (int)l_x0.size();
        int mat0 = pd.ce ? (int)mc_off.size() : (int)m_G.size();
        int nuc0 = (int)n_A.size();
        P.cell0 = (int)c_univ.size();
        P.mat0 = mat0;
        P.root_univ = univ0;
        P.lattice0 = pd.lats.empty() ? -1 : lat0;
        P.ce = pd.ce;
        P.G = pd.G;
        for (size_t i = 0; i < pd.s_type.size(); i++) {
            s_type.push_back(pd.s_type[i]);
            s_bc.push_back(pd.s_bc[i]);
            for (int k = 0; k < 4; k++) s_coef.push_back(pd.s_coef[4 * i + k]);
            double R = pd.s_type[i] == SURF_CYLZ ? pd.s_coef[4 * i + 2]
                     : pd.s_type[i] == SURF_SPHERE ? pd.s_coef[4 * i + 3] : 0.0;
            s_r2.push_back(R * R);
            // z-cylinder on the axis (centre coordinates +0.0): x - 0.0 == x for
            // every x, so the distance code skips those subtractions
            uint64_t c0, c1;
            std::memcpy(&c0, &pd.s_coef[4 * i], 8);
            std::memcpy(&c1, &pd.s_coef[4 * i + 1], 8);
            s_zc.push_back(pd.s_type[i] == SURF_CYLZ && c0 == 0 && c1 == 0 ? 1 : 0);
        }
        int nu = 0;
        for (auto &c : pd.cells) nu = std::max(nu, c.univ + 1);
        for (auto &c : pd.cells) {
            c_univ.push_back(c.univ + univ0);
            c_off.push_back((int)hs_surf.size());
            c_nhs.push_back((int)c.surf.size());
            c_fillk.push_back(c.fillk);
            c_fill.push_back(c.fillk == FILL_MAT ? c.fill + mat0 : c.fill + lat0);
            for (size_t h = 0; h < c.surf.size(); h++) {
                hs_surf.push_back(c.surf[h] + surf0);
                hs_sense.push_back(c.sense[h]);
            }
        }
        for (auto &L : pd.lats) {
            l_x0.push_back(L.x0);
            l_y0.push_back(L.y0);
            l_pitch.push_back(L.pitch);
            l_nx.push_back(L.nx);
            l_ny.push_back(L.ny);
            l_uoff.push_back((int)l_univ.size());
            for (int u : L.univ) l_univ.push_back(u + univ0);
            l_woff.push_back((int)l_wall.size());
            for (int i = 0; i <= L.nx; i++) {
                l_wall.push_back(L.x0 + (double)i * L.pitch);
                l_ctr.push_back(L.x0 + ((double)i + 0.5) * L.pitch);
            }
            for (int i = 0; i <= L.ny; i++) {
                l_wall.push_back(L.y0 + (double)i * L.pitch);
                l_ctr.push_back(L.y0 + ((double)i + 0.5) * L.pitch);
            }
        }
        nuniv += nu;
        if (!pd.ce) {
            int G = pd.G;
            for (auto &m : pd.mg) {
                m_G.push_back(G);
                m_goff.push_back((int)g_sigt.size());
                m_ggoff.push_back((int)gg_sigs.size());
                int fis = 0;
                std::vector<double> row(G);
                for (int g = 0; g < G; g++) {
                    double st = m.sigt[g], nf = m.nusf[g];
                    double acc = 0.0;
                    for (int h = 0; h < G; h++) acc = acc + m.sigs[g * G + h];
                    g_sigt.push_back(st);
                    g_nusf.push_back(nf);
                    g_stot.push_back(acc);
                    g_mfp.push_back(st > 0.0 ? 1.0 / st : HUGE_VAL);
                    double mu = st > 0.0 ? nf / st : 0.0;
                    g_mu.push_back(mu);
                    double fl = std::floor(mu);
                    g_mufl.push_back(fl);
                    g_mufr.push_back(mu - fl);
                    g_ps.push_back(st > 0.0 ? acc / st : 0.0);
                    for (int h = 0; h < G; h++) gg_sigs.push_back(m.sigs[g * G + h]);
                    if (acc > 0.0) make_cdf(&m.sigs[g * G], G, row.data());
                    else std::fill(row.begin(), row.end(), 1.0);
                    for (int h = 0; h < G; h++) gg_scdf.push_back(row[h]);
                    if (nf > 0.0) fis = 1;
                }
                double csum = 0.0;
                for (int g = 0; g < G; g++) csum += m.chi[g];
                if (csum > 0.0) make_cdf(m.chi.data(), G, row.data());
                else std::fill(row.begin(), row.end(), 1.0);
                for (int g = 0; g < G; g++) g_chicdf.push_back(row[g]);
                m_fissile.push_back(fis);
            }
        } else {
            for (auto &u : pd.nucs) {
                nucs.push_back(&u);
                n_A.push_back(u.A);
                n_nu.push_back(u.nu);
                // kinematics: A, 2A, A^2 + 1 (one rounding), 1/(A + 1)^2, 1/(A + 1), 1/A
                const double A1 = u.A + 1.0, A1sq = A1 * A1;
                n_kin.insert(n_kin.end(), {u.A, 2.0 * u.A, std::fma(u.A, u.A, 1.0), 1.0 / A1sq,
                                           1.0 / A1, 1.0 / u.A});
            }
            for (auto &m : pd.mce) {
                mc_off.push_back((int)mc_nuc.size());
                mc_n.push_back((int)m.nuc.size());
                int fis = 0;
                for (size_t k = 0; k < m.nuc.size(); k++) {
                    mc_nuc.push_back(m.nuc[k] + nuc0);
                    mc_dens.push_back(m.dens[k]);
                    const NucDef &u = pd.nucs[m.nuc[k]];
                    if (u.nu > 0.0)
                        for (double f : u.f)
                            if (f > 0.0) {
                                fis = 1;
                                break;
                            }
                }
                mc_fissile.push_back(fis);
            }
        }
        P.src_kind = pd.src.kind;
        P.src_accept = pd.src.accept;
        P.src_ekind = pd.src.ekind;
        P.src_dkind = pd.src.dkind;
        std::memcpy(P.src_p, pd.src.p, sizeof P.src_p);
        std::memcpy(P.src_beam, pd.src.beam, sizeof P.src_beam);
        P.src_E = pd.src.E;
        P.src_cdf_off = (int)src_cdf.size();
        P.src_ncdf = (int)pd.src.pdf.size();
        if (!pd.src.pdf.empty()) {
            std::vector<double> cdf(pd.src.pdf.size());
            make_cdf(pd.src.pdf.data(), (int)cdf.size(), cdf.data());
            src_cdf.insert(src_cdf.end(), cdf.begin(), cdf.end());
        }
        P.tally_first = (int)t_filter.size();
        P.tally_count = (int)pd.tallies.size();
        tally_first.push_back(P.tally_first);
        int ncell = (int)pd.cells.size();
        int nmat = pd.ce ? (int)pd.mce.size() : (int)pd.mg.size();
        for (auto &t : pd.tallies) {
            int nb = t.filter == FILTER_CELL ? ncell
                   : t.filter == FILTER_LATTICE ? pd.lats[0].nx * pd.lats[0].ny : nmat;
            int ne = pd.ce ? (int)t.edges.size() - 1 : pd.G;
            t_filter.push_back(t.filter);
            t_nbins.push_back(nb);
            t_ne.push_back(ne);
            t_batches.push_back(r.batches);
            t_off.push_back((int)acc_size);
            int ntb = t.tedges.empty() ? 0 : (int)t.tedges.size() - 1;
            acc_size += (int64_t)r.batches * nb * ne * std::max(ntb, 1);
            t_eoff.push_back((int)t_edges.size());
            t_nedges.push_back((int)t.edges.size());
            t_edges.insert(t_edges.end(), t.edges.begin(), t.edges.end());
            // time edges and 1 / width (1 / (e[k+1] - e[k]), the last entry unused)
            t_ntb.push_back(ntb);
            t_toff.push_back((int)t_tedges.size());
            for (size_t k = 0; k < t.tedges.size(); k++) {
                t_tedges.push_back(t.tedges[k]);
                t_tinvw.push_back(k + 1 < t.tedges.size() ? 1.0 / (t.tedges[k + 1] - t.tedges[k]) : 0.0);
            }
        }
        if (acc_size > (int64_t)1 << 30) return "tally accumulators too large";
        P.max_coll = pd.max_coll;
        P.fg_kT = pd.fg_kT;
        P.fg_emax = (pd.fg_cut > 0.0 ? pd.fg_cut : 400.0) * pd.fg_kT;
        P.fg_ikT = pd.fg_kT > 0.0 ? 1.0 / pd.fg_kT : 0.0;
        P.time_on = pd.time_on ? 1 : 0;
        P.t0 = pd.t0;
        P.tcut = pd.tcut;
        P.invv_off = (int)g_invv.size();
        if (pd.time_on && !pd.ce) g_invv.insert(g_invv.end(), pd.invv.begin(), pd.invv.end());
        P.batches = r.batches;
        P.seed = r.seed & 0x7FFFFFFFFFFFFFFFULL;
        P.n = r.n;
        probs.push_back(P);
    }

    // universes: cells in definition order
    std::vector<int> u_off(nuniv + 1, 0), u_cells(c_univ.size());
    for (int u : c_univ) u_off[u + 1]++;
    for (int u = 0; u < nuniv; u++) u_off[u + 1] += u_off[u];
    {
        std::vector<int> fill(nuniv, 0);
        for (size_t c = 0; c < c_univ.size(); c++) u_cells[u_off[c_univ[c]] + fill[c_univ[c]]++] = (int)c;
    }
    // Edge cell of each universe: the cell holding every point of a lattice
    // element's boundary, when that can be proven: all of the universe's
    // surfaces are z-cylinders or spheres strictly inside the element of every
    // lattice using it (margin 1e-6 pitch), so f > 0 on the boundary, every
    // half-space there has sense +1 and the first cell (definition order) whose
    // half-spaces are all + is what the full search returns.  -1 otherwise.
    std::vector<int> u_edge(nuniv, -1);
    // c_inner: a universe cell inside (sense -1) a cylinder or sphere that lies
    // strictly inside every lattice element holding the universe (same margin):
    // a particle there leaves that surface before it can reach a lattice wall,
    // so those distances never win and are not computed (root surfaces are
    // skipped only where c_rootfar below proves it too).
    std::vector<int> c_inner(c_univ.size(), 0);
    {
        std::vector<double> upitch(nuniv, 0.0);   // smallest pitch of a lattice using U
        for (size_t L = 0; L < l_pitch.size(); L++) {
            int b = l_uoff[L], e = b + l_nx[L] * l_ny[L];
            for (int k = b; k < e; k++) {
                int U = l_univ[k];
                if (upitch[U] == 0.0 || l_pitch[L] < upitch[U]) upitch[U] = l_pitch[L];
            }
        }
        for (int U = 0; U < nuniv; U++) {
            if (upitch[U] <= 0.0) continue;
            double half = 0.5 * upitch[U] * (1.0 - 1e-6);
            bool ok = true;
            for (int k = u_off[U]; k < u_off[U + 1] && ok; k++) {
                int c = u_cells[k];
                for (int h = 0; h < c_nhs[c] && ok; h++) {
                    int sid = hs_surf[c_off[c] + h];
                    const double *cf = &s_coef[4 * sid];
                    if (s_type[sid] == SURF_CYLZ)
                        ok = std::fabs(cf[0]) + cf[2] < half && std::fabs(cf[1]) + cf[2] < half;
                    else if (s_type[sid] == SURF_SPHERE)
                        ok = std::fabs(cf[0]) + cf[3] < half && std::fabs(cf[1]) + cf[3] < half;
                    else
                        ok = false;
                }
            }
            for (int k = u_off[U]; k < u_off[U + 1]; k++) {
                int c = u_cells[k];
                for (int h = 0; h < c_nhs[c]; h++) {
                    int sid = hs_surf[c_off[c] + h];
                    const double *cf = &s_coef[4 * sid];
                    double R = s_type[sid] == SURF_CYLZ ? cf[2] : s_type[sid] == SURF_SPHERE ? cf[3] : -1.0;
                    if (R >= 0.0 && hs_sense[c_off[c] + h] == -1 && std::fabs(cf[0]) + R < half &&
                        std::fabs(cf[1]) + R < half)
                        c_inner[c] = 1;
                }
            }
            if (!ok) continue;
            for (int k = u_off[U]; k < u_off[U + 1]; k++) {
                int c = u_cells[k];
                bool all_plus = true;
                for (int h = 0; h < c_nhs[c]; h++)
                    if (hs_sense[c_off[c] + h] != 1) all_plus = false;
                if (all_plus) {
                    u_edge[U] = c;
                    break;
                }
            }
        }
    }
    // Root cells filled by a lattice whose half-spaces are all x / y planes at
    // least half a pitch outside the lattice's interior walls: from an element
    // that is not on the lattice's outer ring, the next lattice wall towards
    // any of those planes is strictly nearer, so their distances never win.
    // Each such plane gets the side of the lattice it lies on (1: low x,
    // 2: high x, 3: low y, 4: high y), and by the same argument only an element
    // in the outer column or row on that side can reach it first.
    std::vector<int> c_skiproot(c_univ.size(), 0);
    std::vector<int> hs_side(hs_surf.size(), 0);
    for (size_t c = 0; c < c_univ.size(); c++) {
        if (c_fillk[c] != FILL_LAT) continue;
        int L = c_fill[c];
        double x0 = l_x0[L], y0 = l_y0[L], p = l_pitch[L];
        bool ok = c_nhs[c] > 0;
        std::vector<int> side(c_nhs[c], 0);
        for (int h = 0; h < c_nhs[c] && ok; h++) {
            int sid = hs_surf[c_off[c] + h];
            double v = s_coef[4 * sid];
            if (s_type[sid] == SURF_PX) {
                side[h] = v <= x0 + 0.5 * p ? 1 : (v >= x0 + ((double)l_nx[L] - 0.5) * p ? 2 : 0);
            } else if (s_type[sid] == SURF_PY) {
                side[h] = v <= y0 + 0.5 * p ? 3 : (v >= y0 + ((double)l_ny[L] - 0.5) * p ? 4 : 0);
            }
            ok = side[h] != 0;
        }
        c_skiproot[c] = ok ? 1 : 0;
        if (ok)
            for (int h = 0; h < c_nhs[c]; h++) hs_side[c_off[c] + h] = side[h];
    }
    // Root cells filled by a lattice whose half-spaces are all x / y planes
    // lying on or outside the lattice's outer edges (within 1e-7 pitch): a
    // particle in an inner cell (inside a cylinder or sphere at least 5e-7
    // pitch inside its element) leaves that convex surface before it can reach
    // such a plane, so from inner cells of these root cells no root surface
    // is evaluated.  Any other root boundary (a z-plane, a plane cutting the
    // lattice's elements) is evaluated from inner cells as from any other.
    std::vector<int> c_rootfar(c_univ.size(), 0);
    for (size_t c = 0; c < c_univ.size(); c++) {
        if (c_fillk[c] != FILL_LAT) continue;
        int L = c_fill[c];
        double p = l_pitch[L], m = 1e-7 * p;
        double xl = l_x0[L], xh = l_x0[L] + (double)l_nx[L] * p;
        double yl = l_y0[L], yh = l_y0[L] + (double)l_ny[L] * p;
        bool ok = true;
        for (int h = 0; h < c_nhs[c] && ok; h++) {
            int sid = hs_surf[c_off[c] + h];
            double v = s_coef[4 * sid];
            if (s_type[sid] == SURF_PX) ok = v <= xl + m || v >= xh - m;
            else if (s_type[sid] == SURF_PY) ok = v <= yl + m || v >= yh - m;
            else ok = false;
        }
        c_rootfar[c] = ok ? 1 : 0;
    }
    // candidates across each half-space: cells of the same universe bounded by
    // the same surface with the opposite sense, in definition order
    std::map<std::tuple<int, int, int>, std::vector<int>> bysurf;
    for (size_t c = 0; c < c_univ.size(); c++)
        for (int h = 0; h < c_nhs[c]; h++)
            bysurf[std::make_tuple(c_univ[c], hs_surf[c_off[c] + h], hs_sense[c_off[c] + h])]
                .push_back((int)c);
    std::vector<int> hs_coff(hs_surf.size() + 1, 0), hs_cand;
    for (size_t c = 0; c < c_univ.size(); c++)
        for (int h = 0; h < c_nhs[c]; h++) {
            int k = c_off[c] + h;
            auto it = bysurf.find(std::make_tuple(c_univ[c], hs_surf[k], -hs_sense[k]));
            if (it != bysurf.end()) hs_cand.insert(hs_cand.end(), it->second.begin(), it->second.end());
            hs_coff[k + 1] = (int)hs_cand.size();
        }

    // continuous energy: union grid, per-nuclide interval maps and interval data
    std::vector<double> Eu;
    std::vector<int> ukey_lo(2, 0);
    std::vector<int> cm_off, cm_n, cm_nkey, cm_koff, cm_klo;
    std::vector<long long> cm_key0;
    std::vector<double> cm_E, cm_rec;
    long long ukey0 = 0;
    int nukey = 1;
    std::vector<int> umap, n_ivoff;
    std::vector<double> n_iv;
    if (!nucs.empty()) {
        for (auto *u : nucs) Eu.insert(Eu.end(), u->E.begin(), u->E.end());
        std::sort(Eu.begin(), Eu.end());
        Eu.erase(std::unique(Eu.begin(), Eu.end()), Eu.end());
        size_t nuni = Eu.size();
        // bucket index of the union grid: result of the plain search (largest
        // i <= n-2 with Eu[i] <= E, else 0) at each bucket's lower edge
        auto search = [&](double E) {
            int lo = 0, hi = (int)nuni - 1;
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (!(E < Eu[mid])) lo = mid;
                else hi = mid;
            }
            return lo;
        };
        auto bits = [](double x) { long long b; std::memcpy(&b, &x, 8); return b; };
        long long k0 = bits(Eu.front()) >> 44, k1 = bits(Eu.back()) >> 44;
        ukey0 = k0;
        nukey = (int)(k1 - k0 + 1);
        ukey_lo.resize(nukey + 1);
        for (int b = 0; b <= nukey; b++) {
            long long kb = (k0 + b) << 44;
            double edge;
            std::memcpy(&edge, &kb, 8);
            ukey_lo[b] = search(edge);
        }
        umap.resize(nucs.size() * nuni);
        for (size_t q = 0; q < nucs.size(); q++) {
            const NucDef &u = *nucs[q];
            int n = (int)u.E.size();
            n_ivoff.push_back((int)(n_iv.size() / 8));
            for (int j = 0; j + 1 < n; j++) {
                n_iv.push_back(u.E[j]);
                n_iv.push_back(1.0 / (u.E[j + 1] - u.E[j]));
                n_iv.push_back(u.s[j]);
                n_iv.push_back(u.s[j + 1] - u.s[j]);
                n_iv.push_back(u.c[j]);
                n_iv.push_back(u.c[j + 1] - u.c[j]);
                n_iv.push_back(u.f[j]);
                n_iv.push_back(u.f[j + 1] - u.f[j]);
            }
            int j = 0;
            for (size_t k = 0; k < nuni; k++) {
                while (j + 1 < n && u.E[j + 1] <= Eu[k]) j++;
                umap[q * nuni + k] = std::min(j, n - 2);
            }
        }
        // Macroscopic flight cross sections per material, tabulated on the
        // material's own union grid: at each point the per-nuclide lin-lin
        // values (interval = largest j <= n-2 with E_j <= E), summed in the
        // material's order; per interval (E_k, 1/dE_k, St_k, dSt_k, Sf_k, dSf_k)
        // and a bucket index keyed like the global one.
        for (size_t m = 0; m < mc_off.size(); m++) {
            int o = mc_off[m], nn = mc_n[m];
            std::vector<double> G;
            for (int q = 0; q < nn; q++) G.insert(G.end(), nucs[mc_nuc[o + q]]->E.begin(), nucs[mc_nuc[o + q]]->E.end());
            std::sort(G.begin(), G.end());
            G.erase(std::unique(G.begin(), G.end()), G.end());
            int n = (int)G.size();
            std::vector<double> St(n), Sf(n);
            for (int k = 0; k < n; k++) {
                double E = G[k], sigt = 0.0, nusf = 0.0;
                for (int q = 0; q < nn; q++) {
                    const NucDef &u = *nucs[mc_nuc[o + q]];
                    int lo = 0, hi = (int)u.E.size() - 1;
                    while (hi - lo > 1) {
                        int mid = (lo + hi) / 2;
                        if (u.E[mid] <= E) lo = mid;
                        else hi = mid;
                    }
                    double f = (E - u.E[lo]) * (1.0 / (u.E[lo + 1] - u.E[lo]));
                    double ss = u.s[lo] + f * (u.s[lo + 1] - u.s[lo]);
                    double sc = u.c[lo] + f * (u.c[lo + 1] - u.c[lo]);
                    double sf = u.f[lo] + f * (u.f[lo + 1] - u.f[lo]);
                    double st = ss + sc + sf;
                    sigt = sigt + mc_dens[o + q] * st;
                    nusf = nusf + mc_dens[o + q] * (u.nu * sf);
                }
                St[k] = sigt;
                Sf[k] = nusf;
            }
            cm_off.push_back((int)cm_E.size());
            cm_n.push_back(n);
            for (int k = 0; k < n; k++) {
                cm_E.push_back(G[k]);
                bool last = k + 1 >= n;
                cm_rec.push_back(G[k]);
                cm_rec.push_back(last ? 0.0 : 1.0 / (G[k + 1] - G[k]));
                cm_rec.push_back(St[k]);
                cm_rec.push_back(last ? 0.0 : St[k + 1] - St[k]);
                cm_rec.push_back(Sf[k]);
                cm_rec.push_back(last ? 0.0 : Sf[k + 1] - Sf[k]);
            }
            auto gsearch = [&](double E) {
                int lo = 0, hi = n - 1;
                while (hi - lo > 1) {
                    int mid = (lo + hi) >> 1;
                    if (!(E < G[mid])) lo = mid;
                    else hi = mid;
                }
                return lo;
            };
            long long g0 = bits(G.front()) >> 44, g1 = bits(G.back()) >> 44;
            cm_key0.push_back(g0);
            cm_nkey.push_back((int)(g1 - g0 + 1));
            cm_koff.push_back((int)cm_klo.size());
            for (long long b = 0; b <= g1 - g0 + 1; b++) {
                long long kb = (g0 + b) << 44;
                double edge;
                std::memcpy(&edge, &kb, 8);
                cm_klo.push_back(gsearch(edge));
            }
        }
    }
    // log tables: ln c and 1/c of c = 1 + j/256 in fixed point (Q57, Q63 rounded
    // down), and (e - 53) ln 2 in Q57 for the 54 binades of n
    std::vector<int64_t> lnc_q(256), eln2_q(64);
    std::vector<uint64_t> invc_q(256);
    for (int j = 0; j < 256; j++) {
        lnc_q[j] = ln_table_q57(j);
        invc_q[j] = (uint64_t)((((u128)256) << 63) / (u128)(256 + j));
    }
    const int64_t l2 = ln2_q57();
    for (int e = 0; e < 64; e++) eln2_q[e] = (int64_t)(e - 53) * l2;

    int nrep = acc_size > 0 ? (int)std::max<int64_t>(1, std::min<int64_t>(64, (1 << 20) / acc_size)) : 1;

    Staging S;
    size_t o_prob = S.put(probs);
    size_t o_stype = S.put(s_type), o_sbc = S.put(s_bc), o_scoef = S.put(s_coef), o_sr2 = S.put(s_r2),
           o_szc = S.put(s_zc);
    size_t o_cuniv = S.put(c_univ), o_coff = S.put(c_off), o_cnhs = S.put(c_nhs),
           o_cfillk = S.put(c_fillk), o_cfill = S.put(c_fill);
    // a half-space index travels in 24 bits of a pooled particle's event word
    if (hs_surf.size() >= ((size_t)1 << 23)) return "too many half-spaces (at most 8388607)";
    size_t o_hssurf = S.put(hs_surf), o_hssense = S.put(hs_sense), o_hscoff = S.put(hs_coff),
           o_hscand = S.put(hs_cand), o_uoff = S.put(u_off), o_ucells = S.put(u_cells),
           o_uedge = S.put(u_edge), o_cskip = S.put(c_skiproot), o_hsside = S.put(hs_side),
           o_cinner = S.put(c_inner), o_crootfar = S.put(c_rootfar);
    size_t o_lx0 = S.put(l_x0), o_ly0 = S.put(l_y0), o_lp = S.put(l_pitch), o_lnx = S.put(l_nx),
           o_lny = S.put(l_ny), o_luoff = S.put(l_uoff), o_luniv = S.put(l_univ),
           o_lwoff = S.put(l_woff), o_lwall = S.put(l_wall), o_lctr = S.put(l_ctr);
    size_t o_mG = S.put(m_G), o_mgoff = S.put(m_goff), o_mggoff = S.put(m_ggoff),
           o_mfis = S.put(m_fissile);
    size_t o_sigt = S.put(g_sigt), o_mfp = S.put(g_mfp), o_nusf = S.put(g_nusf), o_mu = S.put(g_mu),
           o_mufl = S.put(g_mufl), o_mufr = S.put(g_mufr), o_ps = S.put(g_ps),
           o_stot = S.put(g_stot), o_chicdf = S.put(g_chicdf), o_sigs = S.put(gg_sigs),
           o_scdf = S.put(gg_scdf);
    size_t o_ukey = S.put(ukey_lo);
    size_t o_cmoff = S.put(cm_off), o_cmn = S.put(cm_n), o_cmnkey = S.put(cm_nkey),
           o_cmkoff = S.put(cm_koff), o_cmklo = S.put(cm_klo), o_cmkey0 = S.put(cm_key0),
           o_cmE = S.put(cm_E), o_cmrec = S.put(cm_rec);
    size_t o_Eu = S.put(Eu), o_umap = S.put(umap), o_nivoff = S.put(n_ivoff), o_niv = S.put(n_iv),
           o_nA = S.put(n_A), o_nnu = S.put(n_nu), o_nkin = S.put(n_kin);
    size_t o_mcoff = S.put(mc_off), o_mcn = S.put(mc_n), o_mcnuc = S.put(mc_nuc),
           o_mcfis = S.put(mc_fissile), o_mcdens = S.put(mc_dens);
    size_t o_srccdf = S.put(src_cdf), o_lncq = S.put(lnc_q), o_invcq = S.put(invc_q),
           o_eln2q = S.put(eln2_q);
    size_t o_tf = S.put(t_filter), o_tnb = S.put(t_nbins), o_tne = S.put(t_ne), o_toff = S.put(t_off),
           o_teoff = S.put(t_eoff), o_tned = S.put(t_nedges), o_tbat = S.put(t_batches),
           o_tedges = S.put(t_edges), o_tntb = S.put(t_ntb), o_ttoff = S.put(t_toff),
           o_ttedges = S.put(t_tedges), o_ttinvw = S.put(t_tinvw), o_ginvv = S.put(g_invv);

    if (dw.arena) {
        cudaFree(dw.arena);
        dw.arena = nullptr;
    }
    cudaError_t e = cudaMalloc(&dw.arena, S.buf.size());
    if (e != cudaSuccess) return std::string("cudaMalloc(world): ") + cudaGetErrorString(e);
    e = cudaMemcpyAsync(dw.arena, S.buf.data(), S.buf.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return std::string("upload(world): ") + cudaGetErrorString(e);
    dw.bytes = S.buf.size();
    // FNV-1a (64-bit) over 8-byte words, then the tail bytes
    uint64_t fp = 14695981039346656037ULL;
    const size_t nw = S.buf.size() / 8;
    for (size_t k = 0; k < nw; k++) {
        uint64_t w;
        std::memcpy(&w, S.buf.data() + 8 * k, 8);
        fp = (fp ^ w) * 1099511628211ULL;
    }
    for (size_t k = 8 * nw; k < S.buf.size(); k++)
        fp = (fp ^ (uint64_t)(unsigned char)S.buf[k]) * 1099511628211ULL;
    dw.fingerprint = fp;
    char *b = (char *)dw.arena;
    World &W = dw.W;
    W.nprob = (int)probs.size();
    W.prob = (const ProblemDev *)(b + o_prob);
#define P_(field, T, off) W.field = (const T *)(b + off)
    P_(s_type, int, o_stype); P_(s_bc, int, o_sbc); P_(s_coef, double, o_scoef); P_(s_r2, double, o_sr2);
    P_(s_zc, int, o_szc);
    P_(c_univ, int, o_cuniv); P_(c_off, int, o_coff); P_(c_nhs, int, o_cnhs);
    P_(c_fillk, int, o_cfillk); P_(c_fill, int, o_cfill);
    P_(hs_surf, int, o_hssurf); P_(hs_sense, int, o_hssense); P_(hs_coff, int, o_hscoff);
    P_(hs_cand, int, o_hscand); P_(u_off, int, o_uoff); P_(u_cells, int, o_ucells); P_(u_edge, int, o_uedge);
    P_(c_skiproot, int, o_cskip);
    P_(hs_side, int, o_hsside);
    P_(c_inner, int, o_cinner);
    P_(c_rootfar, int, o_crootfar);
    P_(l_x0, double, o_lx0); P_(l_y0, double, o_ly0); P_(l_pitch, double, o_lp);
    P_(l_nx, int, o_lnx); P_(l_ny, int, o_lny); P_(l_uoff, int, o_luoff); P_(l_univ, int, o_luniv);
    P_(l_woff, int, o_lwoff); P_(l_wall, double, o_lwall); P_(l_ctr, double, o_lctr);
    P_(m_G, int, o_mG); P_(m_goff, int, o_mgoff); P_(m_ggoff, int, o_mggoff); P_(m_fissile, int, o_mfis);
    P_(g_sigt, double, o_sigt); P_(g_mfp, double, o_mfp); P_(g_nusf, double, o_nusf);
    P_(g_mu, double, o_mu); P_(g_mufl, double, o_mufl); P_(g_mufr, double, o_mufr);
    P_(g_ps, double, o_ps); P_(g_stot, double, o_stot); P_(g_chicdf, double, o_chicdf);
    P_(gg_sigs, double, o_sigs); P_(gg_scdf, double, o_scdf);
    P_(ukey_lo, int, o_ukey);
    P_(cm_off, int, o_cmoff); P_(cm_n, int, o_cmn); P_(cm_nkey, int, o_cmnkey);
    P_(cm_koff, int, o_cmkoff); P_(cm_klo, int, o_cmklo); P_(cm_key0, long long, o_cmkey0);
    P_(cm_E, double, o_cmE); P_(cm_rec, double, o_cmrec);
    P_(Eu, double, o_Eu); P_(umap, int, o_umap); P_(n_ivoff, int, o_nivoff); P_(n_iv, double, o_niv);
    P_(n_A, double, o_nA); P_(n_nu, double, o_nnu); P_(n_kin, double, o_nkin);
    P_(mc_off, int, o_mcoff); P_(mc_n, int, o_mcn); P_(mc_nuc, int, o_mcnuc);
    P_(mc_fissile, int, o_mcfis); P_(mc_dens, double, o_mcdens);
    P_(src_cdf, double, o_srccdf); P_(lnc_q, int64_t, o_lncq); P_(invc_q, uint64_t, o_invcq);
    P_(eln2_q, int64_t, o_eln2q);
    P_(t_filter, int, o_tf); P_(t_nbins, int, o_tnb); P_(t_ne, int, o_tne); P_(t_off, int, o_toff);
    P_(t_eoff, int, o_teoff); P_(t_nedges, int, o_tned); P_(t_batches, int, o_tbat);
    P_(t_edges, double, o_tedges);
    P_(t_ntb, int, o_tntb); P_(t_toff, int, o_ttoff); P_(t_tedges, double, o_ttedges);
    P_(t_tinvw, double, o_ttinvw); P_(g_invv, double, o_ginvv);
#undef P_
    // CE speed: v = kv sqrt(E / 1 eV) cm/s, kv = sqrt(2 e / m_n) * 100
    W.kv = std::sqrt(2.0 * 1.602176634e-19 / 1.67492749804e-27) * 100.0;
    W.time_any = 0;
    for (const ProblemDev &P : probs)
        if (P.time_on) W.time_any = 1;
    for (int n : t_ntb)
        if (n > 0) W.time_any = 1;
    W.ce_any = 0;
    for (const ProblemDev &P : probs)
        if (P.ce) W.ce_any = 1;
    W.need_iw = 0;
    for (int t : s_type)
        if (t == SURF_PZ) W.need_iw = 1;
    W.nunion = (int)Eu.size();
    W.ukey0 = ukey0;
    W.nukey = nukey;
    W.nnuc = (int)nucs.size();
    W.acc_size = (int)acc_size;
    W.nrep = nrep;
    dw.probs = probs;
    dw.tally_first = tally_first;
    dw.t_off = t_off;
    dw.t_nbins = t_nbins;
    dw.t_ne = t_ne;
    dw.t_batches = t_batches;
    dw.t_ntb = t_ntb;
    dw.acc_size = (int)acc_size;
    dw.nrep = nrep;
    return "";
}

}  // namespace mcgb
