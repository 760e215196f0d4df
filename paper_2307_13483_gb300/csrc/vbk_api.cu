// C ABI entry points, model builder, observables (T, sigma, EELS) and the adjoint gradient.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>

#include "vbk_internal.cuh"

static thread_local std::string g_last_error;

void vbk_set_error(const std::string& msg) { g_last_error = msg; }

int vbk_cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
        cudaGetLastError();
        return VBK_ERR_OOM;
    }
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return VBK_ERR_CUDA;
}

namespace {

constexpr int TPB = 256;
inline unsigned cdiv_u(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

int invalid(const std::string& msg) {
    g_last_error = msg;
    return VBK_ERR_INVALID_ARG;
}

// Banded representation of the truncated matrix power (PqP)^k: pw[off][n] = (q^k)_{n, n + off - k}.
std::vector<std::vector<double>> q_power_band(int n, int k) {
    std::vector<std::vector<double>> cur(1, std::vector<double>(n, 1.0));  // identity, k = 0
    for (int kk = 1; kk <= k; ++kk) {
        std::vector<std::vector<double>> nxt(2 * kk + 1, std::vector<double>(n, 0.0));
        // (P q)[r][r+delta] = P[r][r+delta-1] q[r+delta-1][r+delta] + P[r][r+delta+1] q[r+delta+1][r+delta]
        // with q[a][a+1] = q[a+1][a] = sqrt((a+1)/2)
        for (int off = 0; off <= 2 * kk; ++off) {
            const int delta = off - kk;
            for (int r = 0; r < n; ++r) {
                const int col = r + delta;
                if (col < 0 || col >= n) continue;
                double v = 0.0;
                const int c1 = col - 1;  // P[r][col-1] * q[col-1][col]
                if (c1 >= 0) {
                    const int o1 = c1 - r + (kk - 1);
                    if (o1 >= 0 && o1 <= 2 * (kk - 1)) v += cur[o1][r] * std::sqrt((c1 + 1) / 2.0);
                }
                const int c2 = col + 1;  // P[r][col+1] * q[col+1][col]
                if (c2 < n) {
                    const int o2 = c2 - r + (kk - 1);
                    if (o2 >= 0 && o2 <= 2 * (kk - 1)) v += cur[o2][r] * std::sqrt((col + 1) / 2.0);
                }
                nxt[off][r] = v;
            }
        }
        cur.swap(nxt);
    }
    return cur;
}

// The conditions on a model description that need no device, checked before the device is
// touched (so that a malformed description is reported as such on any machine); build() relies
// on them and repeats them where it derives its tables.
int validate_desc(const vbk_model_desc* d) {
    if (!d) return invalid("model description is NULL");
    if (d->n_states < 1 || d->n_states > VBK_MAX_STATES) return invalid("n_states out of range");
    if (d->n_modes < 1 || d->n_modes > VBK_MAX_MODES) return invalid("n_modes out of range");
    long long nnu = 1;
    for (int k = 0; k < d->n_modes; ++k) {
        if (d->n_basis[k] < 1 || d->n_basis[k] > 100000) return invalid("n_basis out of range");
        if (!(d->omega[k] > 0.0) || !std::isfinite(d->omega[k])) return invalid("omega must be positive and finite");
        nnu *= d->n_basis[k];
        if (nnu * d->n_states > (1LL << 30)) return invalid("basis too large");
    }
    if (d->n_terms < 0 || (d->n_terms > 0 && !d->terms)) return invalid("terms missing");
    if (d->n_channels < 1 || d->n_channels > VBK_MAX_CHANNELS || !d->channels) return invalid("n_channels out of range");
    if (d->n_cterms < 0 || d->n_cterms > VBK_MAX_CTERMS || (d->n_cterms > 0 && !d->cterms))
        return invalid("n_cterms out of range (0..VBK_MAX_CTERMS) or cterms missing");
    for (int k = 0; k < d->n_terms; ++k) {
        const vbk_term& t = d->terms[k];
        if (t.d < 0 || t.dp < 0 || t.d >= d->n_states || t.dp >= d->n_states || t.d > t.dp)
            return invalid("term state indices must satisfy 0 <= d <= dp < n_states");
        if (!std::isfinite(t.coef)) return invalid("term coefficient not finite");
        for (int q = 0; q < VBK_MAX_MODES; ++q) {
            if (q < d->n_modes ? (t.pow[q] < 0 || t.pow[q] > 8) : t.pow[q] != 0)
                return invalid("term power out of range (0..8, zero beyond n_modes)");
            if (q < d->n_modes ? (t.raise[q] < 0 || t.raise[q] > 8 || t.lower[q] < 0 || t.lower[q] > 8)
                               : (t.raise[q] != 0 || t.lower[q] != 0))
                return invalid("ladder powers out of range (0..8, zero beyond n_modes)");
            if ((t.raise[q] || t.lower[q]) && t.pow[q])
                return invalid("a mode of a term carries a power of q or a ladder monomial, not both");
        }
    }
    bool seen[MAXS][VBK_MAX_CHANNELS] = {};
    int cnt[VBK_MAX_CHANNELS] = {0}, q_dep[VBK_MAX_CHANNELS] = {0};
    for (int k = 0; k < d->n_channels; ++k) {
        const vbk_channel& c = d->channels[k];
        if (c.d < 0 || c.d >= d->n_states) return invalid("channel state index out of range");
        if (c.mu < 0 || c.mu >= VBK_MAX_CHANNELS) return invalid("partial-wave index out of range");
        if (!(c.a >= 0.0) || !std::isfinite(c.a) || !(c.b > 0.0) || !std::isfinite(c.b) || c.l < 0 || c.l > 20)
            return invalid("channel parameters out of range (a >= 0, b > 0, 0 <= l <= 20)");
        if (seen[c.d][c.mu]) return invalid("a state couples to a partial wave at most once");
        seen[c.d][c.mu] = true;
        if (++cnt[c.mu] > 1) q_dep[c.mu] = 1;
    }
    for (int k = 0; k < d->n_cterms; ++k) {
        const vbk_cterm& t = d->cterms[k];
        if (t.channel < 0 || t.channel >= d->n_channels) return invalid("coupling term names no channel");
        if (!std::isfinite(t.coef)) return invalid("coupling term coefficient not finite");
        for (int q = 0; q < VBK_MAX_MODES; ++q)
            if (q < d->n_modes ? (t.pow[q] < 0 || t.pow[q] > 8) : t.pow[q] != 0)
                return invalid("coupling term power out of range (0..8, zero beyond n_modes)");
        q_dep[d->channels[t.channel].mu] = 1;
    }
    for (int a = 0; a < d->n_channels; ++a)
        for (int b = 0; b < d->n_channels; ++b) {
            const vbk_channel &ca = d->channels[a], &cb = d->channels[b];
            if (ca.mu == cb.mu && q_dep[ca.mu] && ca.l != cb.l)
                return invalid("the channels of a q-dependent partial wave must share l");
        }
    return VBK_OK;
}

int build(const vbk_model_desc* d, vbk_model* m) {
    if (!d) return invalid("model description is NULL");
    if (d->n_states < 1 || d->n_states > VBK_MAX_STATES) return invalid("n_states out of range");
    if (d->n_modes < 1 || d->n_modes > VBK_MAX_MODES) return invalid("n_modes out of range");
    long long nnu = 1;
    for (int k = 0; k < d->n_modes; ++k) {
        if (d->n_basis[k] < 1 || d->n_basis[k] > 100000) return invalid("n_basis out of range");
        if (!(d->omega[k] > 0.0) || !std::isfinite(d->omega[k])) return invalid("omega must be positive and finite");
        nnu *= d->n_basis[k];
    }
    if (nnu * d->n_states > (1LL << 30)) return invalid("basis too large");
    if (d->n_terms < 0 || (d->n_terms > 0 && !d->terms)) return invalid("terms missing");
    if (d->n_channels < 1 || d->n_channels > VBK_MAX_CHANNELS || !d->channels) return invalid("n_channels out of range");
    m->ns = d->n_states;
    m->M = d->n_modes;
    m->Nnu = (int)nnu;
    m->N = (int)(nnu * d->n_states);
    int str = 1;
    for (int k = m->M - 1; k >= 0; --k) {
        m->nb[k] = d->n_basis[k];
        m->stride[k] = str;
        str *= d->n_basis[k];
    }
    if (d->n_cterms < 0 || d->n_cterms > VBK_MAX_CTERMS || (d->n_cterms > 0 && !d->cterms))
        return invalid("n_cterms out of range (0..VBK_MAX_CTERMS) or cterms missing");
    m->terms.assign(d->terms, d->terms + d->n_terms);
    m->chans.assign(d->channels, d->channels + d->n_channels);
    m->cterms.assign(d->cterms, d->cterms + d->n_cterms);
    int mu_d[VBK_MAX_CHANNELS], mu_cnt[VBK_MAX_CHANNELS] = {0}, mu_sw[VBK_MAX_CHANNELS] = {0};
    bool dmu_seen[MAXS][VBK_MAX_CHANNELS] = {};
    for (int k = 0; k < VBK_MAX_CHANNELS; ++k) mu_d[k] = -1;
    int nmu = 0;
    for (const auto& c : m->chans) {
        if (c.d < 0 || c.d >= m->ns) return invalid("channel state index out of range");
        if (c.mu < 0 || c.mu >= VBK_MAX_CHANNELS) return invalid("partial-wave index out of range");
        if (!(c.a >= 0.0) || !std::isfinite(c.a) || !(c.b > 0.0) || !std::isfinite(c.b) || c.l < 0 || c.l > 20)
            return invalid("channel parameters out of range (a >= 0, b > 0, 0 <= l <= 20)");
        if (dmu_seen[c.d][c.mu]) return invalid("a state couples to a partial wave at most once");
        dmu_seen[c.d][c.mu] = true;
        mu_d[c.mu] = c.d;
        mu_cnt[c.mu] += 1;
        nmu = std::max(nmu, c.mu + 1);
    }
    m->nmu = nmu;
    int kmax[MAXM] = {0};
    // q-dependent couplings (Sec. II.C): a wave with two or more states, or a coupling polynomial
    for (const auto& t : m->cterms) {
        if (t.channel < 0 || t.channel >= (int)m->chans.size()) return invalid("coupling term names no channel");
        if (!std::isfinite(t.coef)) return invalid("coupling term coefficient not finite");
        for (int k = 0; k < m->M; ++k) {
            if (t.pow[k] < 0 || t.pow[k] > 8) return invalid("coupling term power out of range (0..8)");
            kmax[k] = std::max(kmax[k], t.pow[k]);
        }
        for (int k = m->M; k < VBK_MAX_MODES; ++k)
            if (t.pow[k] != 0) return invalid("coupling term power given for a mode beyond n_modes");
        mu_sw[m->chans[t.channel].mu] = 1;
    }
    for (int mu = 0; mu < VBK_MAX_CHANNELS; ++mu)
        if (mu_cnt[mu] > 1) mu_sw[mu] = 1;
    for (const auto& c : m->chans)
        for (const auto& c2 : m->chans)
            if (c.mu == c2.mu && mu_sw[c.mu] && c.l != c2.l)
                return invalid("the channels of a q-dependent partial wave must share l");
    for (int mu = 0; mu < VBK_MAX_CHANNELS; ++mu)
        if (mu_sw[mu]) mu_d[mu] = -1;
    for (const auto& t : m->terms) {
        if (t.d < 0 || t.dp < 0 || t.d >= m->ns || t.dp >= m->ns || t.d > t.dp) return invalid("term state indices must satisfy 0 <= d <= dp < n_states");
        if (!std::isfinite(t.coef)) return invalid("term coefficient not finite");
        for (int k = 0; k < m->M; ++k) {
            if (t.pow[k] < 0 || t.pow[k] > 8) return invalid("term power out of range (0..8)");
            if (t.raise[k] < 0 || t.raise[k] > 8 || t.lower[k] < 0 || t.lower[k] > 8)
                return invalid("ladder powers out of range (0..8)");
            if ((t.raise[k] || t.lower[k]) && t.pow[k]) return invalid("a mode of a term carries a power of q or a ladder monomial, not both");
            kmax[k] = std::max(kmax[k], t.pow[k]);
        }
        for (int k = m->M; k < VBK_MAX_MODES; ++k)
            if (t.pow[k] != 0 || t.raise[k] != 0 || t.lower[k] != 0) return invalid("power given for a mode beyond n_modes");
    }
    // tables: for every mode and power k = 1..kmax[m], columns o = 0..k of length n_m
    m->tab.clear();
    m->colbase.assign(m->M, std::vector<int>());
    for (int mm = 0; mm < m->M; ++mm) {
        m->colbase[mm].assign(kmax[mm] + 1, -1);
        for (int k = 1; k <= kmax[mm]; ++k) {
            auto band = q_power_band(m->nb[mm], k);
            m->colbase[mm][k] = (int)m->tab.size();
            for (int o = 0; o <= k; ++o) {
                const int off = 2 * o;  // delta = -k + 2 o  ->  band index delta + k
                for (int n = 0; n < m->nb[mm]; ++n) m->tab.push_back(band[off][n]);
            }
        }
    }
    // ladder monomials (a^+)^j a^k of one mode: per (mode, j, k) two columns of length n_m, the
    // entries a point reads at output level n: T_{n, n + k - j} (the term) and T_{n + j - k, n}
    // (its transpose), with <c - k + j|T|c> = sqrt(c! / (c - k)!) sqrt((c - k + j)! / (c - k)!)
    // for c >= k and c - k + j < n_m (products of truncated matrices), zero otherwise
    std::map<std::tuple<int, int, int>, int> ladder_col;
    auto ladder_entry = [&](int nm, int j, int k, int c) {  // <c - k + j|T|c>
        const int r = c - k + j;
        if (c < k || c >= nm || r < 0 || r >= nm) return 0.0;
        double v = 1.0;
        for (int i = 0; i < k; ++i) v *= std::sqrt((double)(c - i));
        for (int i = 1; i <= j; ++i) v *= std::sqrt((double)(c - k + i));
        return v;
    };
    for (const auto& t : m->terms)
        for (int mm = 0; mm < m->M; ++mm) {
            const int j = t.raise[mm], k = t.lower[mm];
            if (!j && !k) continue;
            const auto key = std::make_tuple(mm, j, k);
            if (ladder_col.count(key)) continue;
            ladder_col[key] = (int)m->tab.size();
            for (int n = 0; n < m->nb[mm]; ++n) m->tab.push_back(ladder_entry(m->nb[mm], j, k, n + k - j));  // T
            for (int n = 0; n < m->nb[mm]; ++n) m->tab.push_back(ladder_entry(m->nb[mm], j, k, n));          // T^T
        }
    if (m->tab.empty()) m->tab.push_back(0.0);
    // stencil points
    std::vector<HostEntry> offd, diagp;
    for (int ti = 0; ti < (int)m->terms.size(); ++ti) {
        const auto& t = m->terms[ti];
        bool ladder = false;
        for (int mm = 0; mm < m->M; ++mm) ladder = ladder || t.raise[mm] || t.lower[mm];
        if (ladder) {
            // points of T (and of T^T): every combination of the q-power offsets, the single
            // offset of each ladder monomial
            int cnt[MAXM], o[MAXM];
            long long ncomb = 1;
            for (int k = 0; k < m->M; ++k) {
                cnt[k] = t.pow[k] + 1;
                ncomb *= cnt[k];
            }
            for (int tr = 0; tr < 2; ++tr)
                for (long long c = 0; c < ncomb; ++c) {
                    long long rem = c;
                    for (int k = m->M - 1; k >= 0; --k) {
                        o[k] = (int)(rem % cnt[k]);
                        rem /= cnt[k];
                    }
                    DevEntry e{};
                    e.lin = 0;
                    bool zero = true;
                    for (int k = 0; k < MAXM; ++k) {
                        e.col[k] = -1;
                        e.delta[k] = 0;
                    }
                    for (int k = 0; k < m->M; ++k) {
                        const int j = t.raise[k], l = t.lower[k];
                        if (j || l) {
                            e.delta[k] = tr == 0 ? l - j : j - l;
                            e.col[k] = ladder_col[std::make_tuple(k, j, l)] + tr * m->nb[k];
                        } else if (t.pow[k]) {
                            e.delta[k] = -t.pow[k] + 2 * o[k];
                            e.col[k] = m->colbase[k][t.pow[k]] + o[k] * m->nb[k];
                        } else {
                            continue;
                        }
                        e.lin += e.delta[k] * m->stride[k];
                        if (e.delta[k] != 0) zero = false;
                    }
                    HostEntry h{};
                    h.term = ti;
                    if (t.d == t.dp) {  // the symmetric part: T / 2 and T^T / 2 on state d
                        h.d = t.d;
                        h.mirror = tr;
                        h.w = 0.5;
                        e.dp = t.d;
                        e.coef = 0.5 * t.coef;
                        h.e = e;
                        (zero ? diagp : offd).push_back(h);
                    } else {  // T in block (d, dp), T^T in block (dp, d)
                        h.d = tr == 0 ? t.d : t.dp;
                        h.mirror = tr;
                        e.dp = tr == 0 ? t.dp : t.d;
                        e.coef = t.coef;
                        h.e = e;
                        offd.push_back(h);
                    }
                }
            continue;
        }
        int cnt[MAXM], o[MAXM];
        long long ncomb = 1;
        for (int k = 0; k < m->M; ++k) {
            cnt[k] = t.pow[k] + 1;
            ncomb *= cnt[k];
            o[k] = 0;
        }
        for (long long c = 0; c < ncomb; ++c) {
            long long rem = c;
            for (int k = m->M - 1; k >= 0; --k) {
                o[k] = (int)(rem % cnt[k]);
                rem /= cnt[k];
            }
            DevEntry e{};
            e.coef = t.coef;
            e.lin = 0;
            bool zero = true;
            for (int k = 0; k < MAXM; ++k) {
                e.col[k] = -1;
                e.delta[k] = 0;
            }
            for (int k = 0; k < m->M; ++k) {
                if (t.pow[k] == 0) continue;
                e.delta[k] = -t.pow[k] + 2 * o[k];
                e.col[k] = m->colbase[k][t.pow[k]] + o[k] * m->nb[k];
                e.lin += e.delta[k] * m->stride[k];
                if (e.delta[k] != 0) zero = false;
            }
            if (t.d == t.dp) {
                e.dp = t.d;
                if (zero)
                    diagp.push_back({t.d, ti, 0, e});
                else
                    offd.push_back({t.d, ti, 0, e});
            } else {
                e.dp = t.dp;
                offd.push_back({t.d, ti, 0, e});
                DevEntry em = e;
                em.dp = t.d;
                offd.push_back({t.dp, ti, 1, em});
            }
        }
    }
    auto by_d = [](const HostEntry& a, const HostEntry& b) { return a.d < b.d; };
    std::stable_sort(offd.begin(), offd.end(), by_d);
    std::stable_sort(diagp.begin(), diagp.end(), by_d);
    m->offd = offd;
    m->diagp = diagp;
    for (int st = 0; st < m->ns; ++st) {
        long long np = 0;
        for (const auto& h : offd) np += h.d == st;
        if (np > 256) return (g_last_error = "more than 256 stencil points for one state", VBK_ERR_UNSUPPORTED);
    }
    // device model
    DevModel& dm = m->dm;
    dm = DevModel{};
    dm.ns = m->ns;
    dm.M = m->M;
    dm.Nnu = m->Nnu;
    dm.N = m->N;
    dm.nmu = m->nmu;
    dm.nchan = (int)m->chans.size();
    for (int k = 0; k < MAXM; ++k) dm.fd_nb[k] = make_fastdiv(k < m->M ? m->nb[k] : 1);
    dm.fd_nnu = make_fastdiv(m->Nnu);
    for (int k = 0; k < MAXM; ++k) {
        dm.nb[k] = k < m->M ? m->nb[k] : 1;
        dm.stride[k] = k < m->M ? m->stride[k] : 0;
        dm.omega[k] = k < m->M ? d->omega[k] : 0.0;
    }
    for (int s = 0; s <= MAXS; ++s) {
        dm.ebeg[s] = 0;
        dm.dbeg[s] = 0;
    }
    for (int s = 0; s <= m->ns; ++s) {
        dm.ebeg[s] = (int)(std::lower_bound(offd.begin(), offd.end(), HostEntry{s, 0, 0, {}}, by_d) - offd.begin());
        dm.dbeg[s] = (int)(std::lower_bound(diagp.begin(), diagp.end(), HostEntry{s, 0, 0, {}}, by_d) - diagp.begin());
    }
    for (int s = m->ns + 1; s <= MAXS; ++s) {
        dm.ebeg[s] = dm.ebeg[m->ns];
        dm.dbeg[s] = dm.dbeg[m->ns];
    }
    for (int st = 0; st < MAXS; ++st) {
        dm.lmin[st] = 0;
        dm.lmax[st] = 0;
    }
    for (const auto& h : offd) {
        dm.lmin[h.d] = std::min(dm.lmin[h.d], h.e.lin);
        dm.lmax[h.d] = std::max(dm.lmax[h.d], h.e.lin);
    }
    for (int c = 0; c < dm.nchan; ++c) {
        dm.ch_d[c] = m->chans[c].d;
        dm.ch_mu[c] = m->chans[c].mu;
        dm.ch_l[c] = m->chans[c].l;
        dm.ch_a[c] = m->chans[c].a;
        dm.ch_b[c] = m->chans[c].b;
        dm.ch_sb[c] = std::sqrt(m->chans[c].b);
        dm.ch_isb[c] = 1.0 / dm.ch_sb[c];
        dm.ch_ib[c] = 1.0 / m->chans[c].b;
        const double cv[5] = {dm.ch_a[c], dm.ch_b[c], dm.ch_sb[c], dm.ch_isb[c], dm.ch_ib[c]};
        for (int q = 0; q < 5; ++q) {
            const dflt v = dd_from(cv[q]);
            dm.ch_df[c][q] = make_float2(v.h, v.l);
        }
    }
    for (int k = 0; k < MAXCH; ++k) dm.mu_d[k] = mu_d[k];
    // sandwich channels: points of the coupling polynomials (merged by offset), pair transforms
    std::vector<double> spc;  // [point][nu]
    {
        for (int k = 0; k < MAXCH; ++k) {
            dm.ch_sw[k] = 0;
            dm.mu_sw[k] = mu_sw[k];
            for (int k2 = 0; k2 < MAXCH; ++k2) dm.sc_pair[k][k2] = -1;
        }
        dm.nsc = 0;
        dm.npair = 0;
        int npts = 0;
        dm.sc_pbeg[0] = 0;
        for (int c = 0; c < dm.nchan; ++c) {
            if (!mu_sw[m->chans[c].mu]) continue;
            const int j = dm.nsc++;
            dm.ch_sw[c] = 1;
            dm.sc_ch[j] = c;
            dm.sc_d[j] = m->chans[c].d;
            dm.sc_mu[j] = m->chans[c].mu;
            // columns of P_c keyed by the offset vector; no terms: P_c = 1
            std::vector<std::pair<std::vector<int>, std::vector<double>>> cols;
            auto column = [&](const std::vector<int>& delta) -> std::vector<double>& {
                for (auto& pr : cols)
                    if (pr.first == delta) return pr.second;
                cols.emplace_back(delta, std::vector<double>(m->Nnu, 0.0));
                return cols.back().second;
            };
            bool any = false;
            for (const auto& t : m->cterms) {
                if (t.channel != c) continue;
                any = true;
                int cnt[MAXM], o[MAXM];
                long long ncomb = 1;
                for (int k = 0; k < m->M; ++k) {
                    cnt[k] = t.pow[k] + 1;
                    ncomb *= cnt[k];
                }
                for (long long cb = 0; cb < ncomb; ++cb) {
                    long long rem = cb;
                    for (int k = m->M - 1; k >= 0; --k) {
                        o[k] = (int)(rem % cnt[k]);
                        rem /= cnt[k];
                    }
                    std::vector<int> delta(m->M, 0);
                    for (int k = 0; k < m->M; ++k) delta[k] = t.pow[k] ? -t.pow[k] + 2 * o[k] : 0;
                    std::vector<double>& col = column(delta);
                    for (int nu = 0; nu < m->Nnu; ++nu) {
                        double v = t.coef;
                        for (int mm = 0; mm < m->M && v != 0.0; ++mm) {
                            if (!t.pow[mm]) continue;
                            const int n = (nu / m->stride[mm]) % m->nb[mm];
                            const int nn = n + delta[mm];
                            v = (nn >= 0 && nn < m->nb[mm])
                                    ? v * m->tab[m->colbase[mm][t.pow[mm]] + o[mm] * m->nb[mm] + n]
                                    : 0.0;
                        }
                        col[nu] += v;
                    }
                }
            }
            if (!any) column(std::vector<int>(m->M, 0)).assign(m->Nnu, 1.0);
            for (auto& pr : cols) {
                bool nz = false;
                for (double v : pr.second) nz = nz || v != 0.0;
                if (!nz) continue;
                if (npts >= MAXSP)
                    return (g_last_error = "the coupling polynomials have more than 64 points", VBK_ERR_UNSUPPORTED);
                int lin = 0;
                for (int k = 0; k < m->M; ++k) lin += pr.first[k] * m->stride[k];
                dm.sp_lin[npts++] = lin;
                m->sp_delta.push_back(pr.first);
                spc.insert(spc.end(), pr.second.begin(), pr.second.end());
            }
            dm.sc_pbeg[j + 1] = npts;
        }
        for (int j = 0; j < dm.nsc; ++j)
            for (int j2 = j; j2 < dm.nsc; ++j2) {
                if (dm.sc_mu[j] != dm.sc_mu[j2]) continue;
                if (dm.npair >= MAXPAIR)
                    return (g_last_error = "more than 20 channel pairs of q-dependent partial waves", VBK_ERR_UNSUPPORTED);
                const int p = dm.npair++;
                dm.sc_pair[j][j2] = dm.sc_pair[j2][j] = p;
                const vbk_channel &ca = m->chans[dm.sc_ch[j]], &cb = m->chans[dm.sc_ch[j2]];
                // f_j f_j' = (sqrt(a_j a_j') / 2 pi) eps^(l+1/2) exp(-(b_j + b_j') eps / 2): one-channel form
                dm.pr_l[p] = ca.l;
                dm.pr_a[p] = j == j2 ? ca.a : std::sqrt(ca.a * cb.a);
                dm.pr_b[p] = j == j2 ? ca.b : 0.5 * (ca.b + cb.b);
                dm.pr_sb[p] = std::sqrt(dm.pr_b[p]);
                dm.pr_isb[p] = 1.0 / dm.pr_sb[p];
                dm.pr_ib[p] = 1.0 / dm.pr_b[p];
            }
    }
    // coefficient columns of the stencil points (Sec. III: "all energy factors and square roots can
    // be precalculated")
    const size_t npc = std::max<size_t>(1, offd.size()) * (size_t)m->Nnu;
    std::vector<double> pc(npc, 0.0);
    for (size_t k = 0; k < offd.size(); ++k) {
        const DevEntry& e = offd[k].e;
        for (int nu = 0; nu < m->Nnu; ++nu) {
            double c = e.coef;
            for (int mm = 0; mm < m->M && c != 0.0; ++mm) {
                if (e.col[mm] < 0) continue;
                const int n = (nu / m->stride[mm]) % m->nb[mm];
                const int nn = n + e.delta[mm];
                c = (nn >= 0 && nn < m->nb[mm]) ? c * m->tab[e.col[mm] + n] : 0.0;
            }
            pc[k * m->Nnu + nu] = c;
        }
    }
    // descriptors and primary-mode coefficient rows of the one-block-per-system kernel, the
    // points of each state grouped by primary mode
    std::vector<int4> rdesc;
    std::vector<int4> wdesc;        // the same points for the windowed matvec: (row offset, lin, col2, m2 | dp << 8)
    std::vector<float2> rct, rctd;  // (-c, -c) and the double-float pair (hi, lo) of +c
    std::vector<double> rct64;      // -c in FP64
    int rsec = 0;
    int rhalo = 0, rok = 1;
    for (int d = 0; d < m->ns; ++d) {
        dm.rbeg[d] = (int)rdesc.size();
        for (int mg = 0; mg < MAXM; ++mg) dm.rcnt[d][mg] = 0;
        for (int mg = 0; mg < m->M; ++mg)
            for (size_t k = 0; k < offd.size(); ++k) {
                if (offd[k].d != d) continue;
                const DevEntry& e = offd[k].e;
                int m1 = -1, m2 = 0, col2 = -1, nmodes = 0;
                for (int mm = 0; mm < m->M; ++mm) {
                    if (e.col[mm] < 0) continue;
                    ++nmodes;
                    if (m1 < 0) {
                        m1 = mm;
                    } else if (col2 < 0) {
                        m2 = mm;
                        col2 = e.col[mm];
                    }
                }
                if ((m1 < 0 ? 0 : m1) != mg) continue;
                if (nmodes > 2) rok = 0;
                if (rct.size() & 1) {  // rows start on 16 bytes: four consecutive entries load as two float4
                    rct.push_back(make_float2(0.f, 0.f));
                    rct64.push_back(0.0);
                    rctd.push_back(make_float2(0.f, 0.f));
                }
                const int off = (int)rct.size();
                for (int n = 0; n < m->nb[mg]; ++n) {
                    double c = e.coef;
                    if (m1 >= 0) {
                        const int nn = n + e.delta[m1];
                        c = (nn >= 0 && nn < m->nb[m1]) ? c * m->tab[e.col[m1] + n] : 0.0;
                    }
                    rct.push_back(make_float2((float)-c, (float)-c));
                    rct64.push_back(-c);
                    const float ch = (float)c;
                    rctd.push_back(make_float2(ch, (float)(c - (double)ch)));
                }
                const int poff = (e.dp - d) * m->Nnu + e.lin;
                rdesc.push_back(make_int4(off * 8, poff * 8, col2, m2));
                wdesc.push_back(make_int4(off * 8, e.lin, col2, m2 | (e.dp << 8)));
                if (col2 >= 0) rsec = 1;
                dm.rcnt[d][mg] += 1;
                rhalo = std::max(rhalo, std::max(-(d * m->Nnu + poff), (d + 1) * m->Nnu - 1 + poff - (m->N - 1)));
            }
        if ((int)rdesc.size() - dm.rbeg[d] > 64) rok = 0;
    }
    dm.rbeg[m->ns] = (int)rdesc.size();
    if (rdesc.empty()) rdesc.push_back(make_int4(0, 0, -1, 0));
    if (wdesc.empty()) wdesc.push_back(make_int4(0, 0, -1, 0));
    if (rct.empty()) rct.push_back(make_float2(0.f, 0.f));
    if (rct64.empty()) rct64.push_back(0.0);
    if (rctd.empty()) rctd.push_back(make_float2(0.f, 0.f));
    dm.rsec = rsec;
    if (rdesc.size() > (size_t)MAXS * 64) rok = 0;
    dm.nrct = (int)rct.size();
    dm.rhalo = rhalo;
    dm.rok = rok;
    // energy-independent parts of the diagonal: E_nu per nu and the delta = 0 terms of U_dd per
    // element (the same products as the off-diagonal coefficients, summed in point order)
    std::vector<double> enu(m->Nnu), u0(m->N, 0.0);
    for (int nu = 0; nu < m->Nnu; ++nu) {
        double en = 0.0;
        for (int mm = 0; mm < m->M; ++mm) en += dm.omega[mm] * ((nu / m->stride[mm]) % m->nb[mm] + 0.5);
        enu[nu] = en;
    }
    for (int d = 0; d < m->ns; ++d)
        for (int nu = 0; nu < m->Nnu; ++nu) {
            double u = 0.0;
            for (const HostEntry& h : diagp) {
                if (h.d != d) continue;
                double c = h.e.coef;
                for (int mm = 0; mm < m->M; ++mm)
                    if (h.e.col[mm] >= 0) c *= m->tab[h.e.col[mm] + (nu / m->stride[mm]) % m->nb[mm]];
                u += c;
            }
            u0[(size_t)d * m->Nnu + nu] = u;
        }
    // one device allocation: entries | diagonal entries | tab64 | tab32 | pc64 | pc32 | rdesc | rct
    const size_t ne = std::max<size_t>(1, offd.size()), nd = std::max<size_t>(1, diagp.size()), nt = m->tab.size();
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b1 = al(ne * sizeof(DevEntry)), b2 = al(nd * sizeof(DevEntry)), b3 = al(nt * sizeof(double)),
                 b4 = al(nt * sizeof(float)), b5 = al(npc * sizeof(double)), b6 = al(npc * sizeof(float)),
                 b7 = al(rdesc.size() * sizeof(int4)), b8 = al(rct.size() * sizeof(float2)),
                 b9 = al(npc * sizeof(float2)), b10 = al(rctd.size() * sizeof(float2)),
                 b11 = al(enu.size() * sizeof(double)), b12 = al(u0.size() * sizeof(double)),
                 b13 = al(wdesc.size() * sizeof(int4)), b14 = al(rct64.size() * sizeof(double));
    char* mem = nullptr;
    cudaError_t err =
        cudaMalloc((void**)&mem, b1 + b2 + b3 + b4 + b5 + b6 + b7 + b8 + b9 + b10 + b11 + b12 + b13 + b14);
    if (err != cudaSuccess) return vbk_cuda_fail(err, "model tables");
    m->dev_mem = mem;
    std::vector<DevEntry> he(ne), hd(nd);
    for (size_t k = 0; k < offd.size(); ++k) he[k] = offd[k].e;
    for (size_t k = 0; k < diagp.size(); ++k) hd[k] = diagp[k].e;
    std::vector<float> t32(nt);
    for (size_t k = 0; k < nt; ++k) t32[k] = (float)m->tab[k];
    if ((err = cudaMemcpy(mem, he.data(), ne * sizeof(DevEntry), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (err = cudaMemcpy(mem + b1, hd.data(), nd * sizeof(DevEntry), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (err = cudaMemcpy(mem + b1 + b2, m->tab.data(), nt * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (err = cudaMemcpy(mem + b1 + b2 + b3, t32.data(), nt * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return vbk_cuda_fail(err, "model table upload");
    {
        std::vector<float> pc32(npc);
        for (size_t k = 0; k < npc; ++k) pc32[k] = (float)pc[k];
        if ((err = cudaMemcpy(mem + b1 + b2 + b3 + b4, pc.data(), npc * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (err = cudaMemcpy(mem + b1 + b2 + b3 + b4 + b5, pc32.data(), npc * sizeof(float), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
            return vbk_cuda_fail(err, "model coefficient upload");
        dm.pc64 = (const double*)(mem + b1 + b2 + b3 + b4);
        dm.pc32 = (const float*)(mem + b1 + b2 + b3 + b4 + b5);
    }
    {
        char* base = mem + b1 + b2 + b3 + b4 + b5 + b6;
        if ((err = cudaMemcpy(base, rdesc.data(), rdesc.size() * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (err = cudaMemcpy(base + b7, rct.data(), rct.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
            return vbk_cuda_fail(err, "model descriptor upload");
        dm.rdesc = (const int4*)base;
        dm.rct = (const float2*)(base + b7);
        std::vector<float2> pcs(npc);
        for (size_t k = 0; k < npc; ++k) {
            const float h = (float)pc[k];
            pcs[k] = make_float2(h, (float)(pc[k] - (double)h));
        }
        if ((err = cudaMemcpy(base + b7 + b8, pcs.data(), npc * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
            return vbk_cuda_fail(err, "model coefficient upload");
        dm.pcs = (const float2*)(base + b7 + b8);
        if ((err = cudaMemcpy(base + b7 + b8 + b9, rctd.data(), rctd.size() * sizeof(float2), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return vbk_cuda_fail(err, "model coefficient upload");
        dm.rctd = (const float2*)(base + b7 + b8 + b9);
        char* b2base = base + b7 + b8 + b9 + b10;
        if ((err = cudaMemcpy(b2base, enu.data(), enu.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (err = cudaMemcpy(b2base + b11, u0.data(), u0.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
            return vbk_cuda_fail(err, "model diagonal upload");
        dm.enu = (const double*)b2base;
        dm.u0 = (const double*)(b2base + b11);
        char* b3base = b2base + b11 + b12;
        if ((err = cudaMemcpy(b3base, wdesc.data(), wdesc.size() * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (err = cudaMemcpy(b3base + b13, rct64.data(), rct64.size() * sizeof(double), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
            return vbk_cuda_fail(err, "model descriptor upload");
        dm.wdesc = (const int4*)b3base;
        dm.rct64 = (const double*)(b3base + b13);
    }
    {  // double-float tables of the energy diagonal: Dawson, erfcx, Taylor, u0 per element
        std::vector<float2> dws, erx, tay, u0d(m->N);
        vbk_df_tables(&dws, &erx, &tay);
        for (int i = 0; i < m->N; ++i) {
            const dflt v = dd_from(u0[i]);
            u0d[i] = make_float2(v.h, v.l);
        }
        const size_t c1 = al(dws.size() * sizeof(float2)), c2 = al(erx.size() * sizeof(float2)),
                     c3 = al(tay.size() * sizeof(float2)), c4 = al(u0d.size() * sizeof(float2));
        char* mem3 = nullptr;
        if ((err = cudaMalloc((void**)&mem3, c1 + c2 + c3 + c4)) != cudaSuccess) return vbk_cuda_fail(err, "double-float tables");
        m->dev_mem3 = mem3;
        if ((err = cudaMemcpy(mem3, dws.data(), dws.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (err = cudaMemcpy(mem3 + c1, erx.data(), erx.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (err = cudaMemcpy(mem3 + c1 + c2, tay.data(), tay.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (err = cudaMemcpy(mem3 + c1 + c2 + c3, u0d.data(), u0d.size() * sizeof(float2), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
            return vbk_cuda_fail(err, "double-float table upload");
        dm.dawson_df = (const float2*)mem3;
        dm.erfcx_df = (const float2*)(mem3 + c1);
        dm.taylor_df = (const float2*)(mem3 + c1 + c2);
        dm.u0df = (const float2*)(mem3 + c1 + c2 + c3);
    }
    if (!spc.empty()) {
        const size_t bs = (spc.size() * sizeof(double) + 255) & ~size_t(255);
        char* mem2 = nullptr;
        if ((err = cudaMalloc((void**)&mem2, bs + spc.size() * sizeof(float))) != cudaSuccess)
            return vbk_cuda_fail(err, "coupling polynomial tables");
        m->dev_mem2 = mem2;
        std::vector<float> s32(spc.size());
        for (size_t k = 0; k < spc.size(); ++k) s32[k] = (float)spc[k];
        if ((err = cudaMemcpy(mem2, spc.data(), spc.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (err = cudaMemcpy(mem2 + bs, s32.data(), s32.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
            return vbk_cuda_fail(err, "coupling polynomial upload");
        dm.spc64 = (const double*)mem2;
        dm.spc32 = (const float*)(mem2 + bs);
    }
    dm.ent = (const DevEntry*)mem;
    dm.dent = (const DevEntry*)(mem + b1);
    dm.tab64 = (const double*)(mem + b1 + b2);
    dm.ntab = (int)nt;
    dm.tab32 = (const float*)(mem + b1 + b2 + b3);
    m->desc = *d;
    m->desc.terms = m->terms.data();
    m->desc.channels = m->chans.data();
    m->desc.cterms = m->cterms.empty() ? nullptr : m->cterms.data();
    return VBK_OK;
}

int flat_index(const vbk_model* m, const int* v, int* out) {
    int f = 0;
    for (int k = 0; k < m->M; ++k) {
        if (v[k] < 0 || v[k] >= m->nb[k]) return invalid("vibrational multi-index out of range");
        f += v[k] * m->stride[k];
    }
    *out = f;
    return VBK_OK;
}

double level_energy(const vbk_model* m, const int* v) {
    double e = 0.0;
    for (int k = 0; k < m->M; ++k) e += m->dm.omega[k] * (v[k] + 0.5);
    return e;
}

int check_model(const vbk_model* m) {
    if (!m) return invalid("model handle is NULL");
    return VBK_OK;
}

struct DevBuf {
    void* p = nullptr;
    cudaStream_t st = nullptr;
    ~DevBuf() {
        if (p) cudaFreeAsync(p, st);
    }
};

// --------------------------------------------------------------------------- kernels
// Phi^{v mu} of a q-dependent wave (Sec. II.C, II.D): sum over its channels j of
// f_j(eps) (P_j |v>) in state d_j, i.e. w * f_j * (P_j)_{v + lin_k, v} at v + lin_k for every point
// k of P_j (P_j symmetric), added to the vector g of one system.  The targets are distinct: the
// offsets of one channel differ and the channels of one wave sit in different states.  Returns
// the sum of (f_j (P_j)_{v + lin_k, v})^2, the squared norm of Phi for w = 1.
__device__ double sand_scatter(const DevModel& md, int mu, double eps, int v, double2 w, double2* __restrict__ g) {
    double nrm = 0.0;
    for (int j = 0; j < md.nsc; ++j) {
        if (md.sc_mu[j] != mu) continue;
        const int c = md.sc_ch[j];
        const double f = vbk_amplitude(eps, md.ch_a[c], md.ch_b[c], md.ch_l[c]);
        if (f == 0.0) continue;
        double2* gd = g + (long long)md.sc_d[j] * md.Nnu;
        for (int k = md.sc_pbeg[j]; k < md.sc_pbeg[j + 1]; ++k) {
            const double cf = md.spc64[(long long)k * md.Nnu + v];
            if (cf == 0.0) continue;
            double2& t = gd[v + md.sp_lin[k]];
            t.x += w.x * f * cf;
            t.y += w.y * f * cf;
            nrm += (f * cf) * (f * cf);
        }
    }
    return nrm;
}

// <Phi^{v mu} | psi> of a q-dependent wave: sum_j f_j(eps) (P_j psi_(d_j))(v)  (Eq. crs2, real Phi).
__device__ double2 sand_project(const DevModel& md, int mu, double eps, int v, const double2* __restrict__ ps) {
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < md.nsc; ++j) {
        if (md.sc_mu[j] != mu) continue;
        const int c = md.sc_ch[j];
        const double f = vbk_amplitude(eps, md.ch_a[c], md.ch_b[c], md.ch_l[c]);
        if (f == 0.0) continue;
        const double2* pd = ps + (long long)md.sc_d[j] * md.Nnu;
        double2 t = make_double2(0.0, 0.0);
        for (int k = md.sc_pbeg[j]; k < md.sc_pbeg[j + 1]; ++k) {
            const double cf = md.spc64[(long long)k * md.Nnu + v];
            if (cf == 0.0) continue;
            const double2 x = pd[v + md.sp_lin[k]];
            t.x += cf * x.x;
            t.y += cf * x.y;
        }
        acc.x += f * t.x;
        acc.y += f * t.y;
    }
    return acc;
}

// Dense right-hand sides Phi^{v_i mu} (Sec. II.D): f_{d(mu)}(E - E_vi) on entry (d(mu), v_i), or
// the polynomial columns of a q-dependent wave (Sec. II.C).  b is zero on entry.  bn2[s] receives
// ||Phi||^2 (the sum of the squared entries written), so the solver need not read b for it.
__global__ void k_build_rhs(DevModel md, int nsys, int n_vi, const double* __restrict__ eps, const int* __restrict__ vflat,
                            double2* __restrict__ b, double* __restrict__ bn2) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const int mu = s % md.nmu, i = (s / md.nmu) % n_vi, e = s / (md.nmu * n_vi);
    if (md.mu_sw[mu]) {
        bn2[s] = sand_scatter(md, mu, eps[e], vflat[i], make_double2(1.0, 0.0), b + (long long)s * md.N);
        return;
    }
    const int d = md.mu_d[mu];
    double nrm = 0.0;
    if (d >= 0)
        for (int c = 0; c < md.nchan; ++c)
            if (md.ch_mu[c] == mu) {  // one channel per wave here
                const double f = vbk_amplitude(eps[e], md.ch_a[c], md.ch_b[c], md.ch_l[c]);
                b[(long long)s * md.N + (long long)d * md.Nnu + vflat[i]] = make_double2(f, 0.0);
                nrm = f * f;
            }
    bn2[s] = nrm;
}

__device__ __forceinline__ int chan_of_mu(const DevModel& md, int mu) {
    for (int c = 0; c < md.nchan; ++c)
        if (md.ch_mu[c] == mu) return c;
    return -1;
}

// T_{mu_f vf <- mu_i vi} = f_{mu_f}(E - E_vf) psi_{d(mu_f), vf}  (Eq. crs2 with real Phi);
// sigma = 2 pi^3 / eps_i sum |T|^2 (Eq. crs).  One thread per (e, i, f).
__global__ void k_sigma(DevModel md, int n_eps, int n_vi, int n_vf, const double* __restrict__ eps,
                        const double* __restrict__ Etot, const double2* __restrict__ psi, const int* __restrict__ vf_flat,
                        const double* __restrict__ E_vf, double* __restrict__ sigma, double2* __restrict__ T) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_eps * n_vi * n_vf) return;
    const int f = (int)(t % n_vf), i = (int)((t / n_vf) % n_vi), e = (int)(t / ((long long)n_vf * n_vi));
    const double E = Etot[(long long)e * n_vi + i];
    const int nmu = md.nmu;
    double acc = 0.0;
    for (int mi = 0; mi < nmu; ++mi) {
        const double2* ps = psi + (((long long)e * n_vi + i) * nmu + mi) * (long long)md.N;
        for (int mf = 0; mf < nmu; ++mf) {
            const int d = md.mu_d[mf], c = chan_of_mu(md, mf);
            double2 tv = make_double2(0.0, 0.0);
            if (md.mu_sw[mf]) {
                tv = sand_project(md, mf, E - E_vf[f], vf_flat[f], ps);
            } else if (d >= 0 && c >= 0) {
                const double amp = vbk_amplitude(E - E_vf[f], md.ch_a[c], md.ch_b[c], md.ch_l[c]);
                const double2 pv = ps[(long long)d * md.Nnu + vf_flat[f]];
                tv = make_double2(amp * pv.x, amp * pv.y);
            }
            acc += tv.x * tv.x + tv.y * tv.y;
            if (T) T[((((long long)e * n_vi + i) * nmu + mi) * n_vf + f) * nmu + mf] = tv;
        }
    }
    const double PI = 3.14159265358979323846;
    sigma[t] = 2.0 * PI * PI * PI / eps[e] * acc;
}

// S(eps, de_k) = sum_f sigma_f rho(de_k - (E_vf - E_vi)), rho a unit-area Gaussian (Eq. 2Dsp)
__global__ void k_eels(int n_eps, int n_vi, int n_vf, int n_de, const double* __restrict__ sigma,
                       const double* __restrict__ de, const double* __restrict__ E_vf, const double* __restrict__ E_vi,
                       double sdev, double* __restrict__ S) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_eps * n_vi * n_de) return;
    const int k = (int)(t % n_de), i = (int)((t / n_de) % n_vi), e = (int)(t / ((long long)n_de * n_vi));
    const double* sg = sigma + ((long long)e * n_vi + i) * n_vf;
    const double norm = 1.0 / (sdev * 2.5066282746310002);  // 1 / (s sqrt(2 pi))
    double acc = 0.0;
    for (int f = 0; f < n_vf; ++f) {
        const double x = (de[k] - (E_vf[f] - E_vi[i])) / sdev;
        acc += sg[f] * exp(-0.5 * x * x);
    }
    S[t] = acc * norm;
}

// Adjoint right-hand side per forward system (e, i, mu_i):
//   g = sum_{f, mu_f} w Phi_f^{mu_f},  w = dL/dsigma * 2 pi^3/eps * 2 conj(T)
// and the weights w (stored for the parameter derivatives of Phi_f).
__global__ void k_adjoint_rhs(DevModel md, int n_eps, int n_vi, int n_vf, const double* __restrict__ eps,
                              const double* __restrict__ Etot, const double2* __restrict__ T,
                              const double* __restrict__ dLds, const int* __restrict__ vf_flat, const double* __restrict__ E_vf,
                              double2* __restrict__ g, double2* __restrict__ W) {
    const int nmu = md.nmu;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (long long)n_eps * n_vi * nmu) return;
    const int mi = (int)(s % nmu), i = (int)((s / nmu) % n_vi), e = (int)(s / ((long long)nmu * n_vi));
    const double E = Etot[(long long)e * n_vi + i];
    const double PI = 3.14159265358979323846;
    const double pre = 2.0 * PI * PI * PI / eps[e] * 2.0;
    for (int f = 0; f < n_vf; ++f) {
        const double dl = dLds[((long long)e * n_vi + i) * n_vf + f];
        for (int mf = 0; mf < nmu; ++mf) {
            const double2 tv = T[((((long long)e * n_vi + i) * nmu + mi) * n_vf + f) * nmu + mf];
            const double2 w = make_double2(dl * pre * tv.x, -dl * pre * tv.y);
            W[(s * n_vf + f) * nmu + mf] = w;
            if (md.mu_sw[mf]) {
                sand_scatter(md, mf, E - E_vf[f], vf_flat[f], w, g + s * md.N);
                continue;
            }
            const int d = md.mu_d[mf], c = chan_of_mu(md, mf);
            if (d < 0 || c < 0) continue;
            const double amp = vbk_amplitude(E - E_vf[f], md.ch_a[c], md.ch_b[c], md.ch_l[c]);
            double2& gv = g[s * md.N + (long long)d * md.Nnu + vf_flat[f]];
            gv.x += w.x * amp;
            gv.y += w.y * amp;
        }
    }
}

// Gradient parameter descriptor: kind 0 = term coefficient (points [pb, pe) of the point list),
// kind 1 = channel a, kind 2 = channel b (channel index c), kind 3 = coefficient of a coupling-
// polynomial term of channel c (its unit-coefficient points [pb, pe)).  j = sandwich index of
// channel c (q-dependent coupling, Sec. II.C), -1 for a diagonal channel or a U term.
struct GradParam {
    int kind, c, pb, pe, j;
};

template <int M> __device__ __forceinline__ void decode_nu(const DevModel& md, int nu, int (&n)[MAXM]) {
    int rem = nu;
#pragma unroll
    for (int m = M - 1; m >= 0; --m) {
        n[m] = rem % md.nb[m];
        rem /= md.nb[m];
    }
#pragma unroll
    for (int m = M; m < MAXM; ++m) n[m] = 0;
}

// Element-wise contractions  Re(lambda_i [dA-part psi]_i)  per parameter (see vbk_solve_adjoint);
// part[s][blk][theta].
template <int M>
__global__ void __launch_bounds__(TPB) k_adjoint_contract(DevModel md, int nsys, int n_vi, const double* __restrict__ Etot,
                                                         const double2* __restrict__ lam, const double2* __restrict__ psi,
                                                         int ntheta, const GradParam* __restrict__ gp,
                                                         const int* __restrict__ pt_d, const DevEntry* __restrict__ pts,
                                                         double* __restrict__ part) {
    __shared__ double red[TPB / 32];
    const int s = blockIdx.y;
    const int N = md.N;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nmu = md.nmu;
    const double E = Etot[s / nmu];  // systems are (e, i, mu) with e*n_vi+i = s / nmu
    (void)n_vi;
    int d = 0, nu = 0;
    int n[MAXM];
    double en = 0.0;
    double2 li = make_double2(0.0, 0.0), pi = make_double2(0.0, 0.0);
    const double2* ps = psi + (long long)s * N;
    if (i < N) {
        d = i / md.Nnu;
        nu = i - d * md.Nnu;
        decode_nu<M>(md, nu, n);
#pragma unroll
        for (int m = 0; m < M; ++m) en += md.omega[m] * (n[m] + 0.5);
        li = lam[(long long)s * N + i];
        pi = ps[i];
    }
    for (int th = 0; th < ntheta; ++th) {
        const GradParam g = gp[th];
        double v = 0.0;
        if (i < N) {
            if (g.kind == 0) {
                double2 acc = make_double2(0.0, 0.0);
                for (int k = g.pb; k < g.pe; ++k) {
                    if (pt_d[k] != d) continue;
                    const DevEntry p = pts[k];
                    double c = p.coef;
                    bool ok = true;
#pragma unroll
                    for (int m = 0; m < M; ++m)
                        if (p.col[m] >= 0) {
                            const int nn = n[m] + p.delta[m];
                            ok = ok && nn >= 0 && nn < md.nb[m];
                            c *= md.tab64[p.col[m] + n[m]];
                        }
                    if (ok) {
                        const double2 x = ps[p.dp * md.Nnu + nu + p.lin];
                        acc.x += c * x.x;
                        acc.y += c * x.y;
                    }
                }
                // -lambda^T (dA) psi with dA = -(unit-coefficient term matrix)
                const double2 t = cmul<double>(li, acc);
                v = t.x;
            } else if (g.j < 0 && md.ch_d[g.c] == d) {
                const int c = g.c;
                const double eps = E - en;
                if (g.kind == 1) {  // dA/da = -F/a
                    const double2 F = vbk_level_shift_eval(eps, 1.0, md.ch_b[c], md.ch_l[c]);
                    v = cmul<double>(li, cmul<double>(F, pi)).x;
                } else {  // dA/db = F^{(l+1)}  (the transform with l -> l+1)
                    const double2 F = vbk_level_shift_eval(eps, md.ch_a[c], md.ch_b[c], md.ch_l[c] + 1);
                    v = -cmul<double>(li, cmul<double>(F, pi)).x;
                }
            }
        }
        // block reduction of v
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < TPB / 32; ++w) t += red[w];
            part[((long long)s * gridDim.x + blockIdx.x) * ntheta + th] = t;
        }
    }
}

// Parameter derivatives of the right-hand sides (channel a, b only), one thread per system:
//   Re[ sum_f w_f dPhi_f^T psi + lambda^T dPhi_i ],  dPhi/da = Phi/(2a), dPhi/db = -(eps/2) Phi.
__global__ void k_adjoint_rhs_terms(DevModel md, int n_eps, int n_vi, int n_vf, const double* __restrict__ eps,
                                    const double* __restrict__ Etot, const int* __restrict__ vi_flat,
                                    const double* __restrict__ E_vi, const int* __restrict__ vf_flat,
                                    const double* __restrict__ E_vf, const double2* __restrict__ W,
                                    const double2* __restrict__ lam, const double2* __restrict__ psi, int ntheta,
                                    const GradParam* __restrict__ gp, const DevEntry* __restrict__ pts,
                                    double* __restrict__ out) {
    const int nmu = md.nmu;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (long long)n_eps * n_vi * nmu) return;
    const int mi = (int)(s % nmu), i = (int)((s / nmu) % n_vi), e = (int)(s / ((long long)nmu * n_vi));
    const double E = Etot[(long long)e * n_vi + i];
    const double2* ps = psi + s * md.N;
    const double2* ls = lam + s * md.N;
    for (int th = 0; th < ntheta; ++th) {
        const GradParam g = gp[th];
        double acc = 0.0;
        if (g.j >= 0) {
            // q-dependent channel: Phi^{v mu} carries f_c(eps) P_c |v>, so dPhi = df P_c |v> (kinds 1, 2)
            // or f Q_t |v> (kind 3, Q_t the unit-coefficient term); both sums use (X y_(d_c))(v)
            // for the symmetric operator X = P_c or Q_t
            const int c = g.c, mu = md.ch_mu[c], d = md.ch_d[c], j = g.j;
            const double a = md.ch_a[c], b = md.ch_b[c];
            const int l = md.ch_l[c];
            auto apply = [&](const double2* y, int v) -> double2 {
                double2 t = make_double2(0.0, 0.0);
                const double2* yd = y + (long long)d * md.Nnu;
                if (g.kind == 3) {
                    int n[MAXM];
                    int rem = v;
                    for (int m = md.M - 1; m >= 0; --m) {
                        n[m] = rem % md.nb[m];
                        rem /= md.nb[m];
                    }
                    for (int k = g.pb; k < g.pe; ++k) {
                        const DevEntry pt = pts[k];
                        double cf = 1.0;
                        bool ok = true;
                        for (int m = 0; m < md.M; ++m)
                            if (pt.col[m] >= 0) {
                                const int nn = n[m] + pt.delta[m];
                                ok = ok && nn >= 0 && nn < md.nb[m];
                                cf *= md.tab64[pt.col[m] + n[m]];
                            }
                        if (ok) {
                            const double2 x = yd[v + pt.lin];
                            t.x += cf * x.x;
                            t.y += cf * x.y;
                        }
                    }
                } else {
                    for (int k = md.sc_pbeg[j]; k < md.sc_pbeg[j + 1]; ++k) {
                        const double cf = md.spc64[(long long)k * md.Nnu + v];
                        if (cf == 0.0) continue;
                        const double2 x = yd[v + md.sp_lin[k]];
                        t.x += cf * x.x;
                        t.y += cf * x.y;
                    }
                }
                return t;
            };
            auto dfac = [&](double ep) {  // df/da, df/db, or f itself (kind 3)
                const double f = vbk_amplitude(ep, a, b, l);
                return g.kind == 1 ? (a > 0 ? f / (2.0 * a) : 0.0) : g.kind == 2 ? -0.5 * ep * f : f;
            };
            if (mi == mu) {  // lambda^T dPhi_i
                const double ei = E - E_vi[i];
                acc += dfac(ei) * apply(ls, vi_flat[i]).x;
            }
            for (int f = 0; f < n_vf; ++f) {  // sum_f w_f dPhi_f^T psi
                const double ef = E - E_vf[f];
                const double2 w = W[(s * n_vf + f) * nmu + mu];
                acc += dfac(ef) * cmul<double>(w, apply(ps, vf_flat[f])).x;
            }
        } else if (g.kind != 0) {
            const int c = g.c, mu = md.ch_mu[c], d = md.ch_d[c];
            const double a = md.ch_a[c], b = md.ch_b[c];
            const int l = md.ch_l[c];
            if (mi == mu) {  // lambda^T dPhi_i
                const double ei = E - E_vi[i];
                const double f = vbk_amplitude(ei, a, b, l);
                const double df = g.kind == 1 ? (a > 0 ? f / (2.0 * a) : 0.0) : -0.5 * ei * f;
                acc += df * ls[(long long)d * md.Nnu + vi_flat[i]].x;
            }
            for (int f = 0; f < n_vf; ++f) {  // sum_f w_f dPhi_f^T psi
                const double ef = E - E_vf[f];
                const double fa = vbk_amplitude(ef, a, b, l);
                const double df = g.kind == 1 ? (a > 0 ? fa / (2.0 * a) : 0.0) : -0.5 * ef * fa;
                const double2 w = W[(s * n_vf + f) * nmu + mu];
                const double2 pv = ps[(long long)d * md.Nnu + vf_flat[f]];
                acc += df * cmul<double>(w, pv).x;
            }
        }
        out[s * ntheta + th] = acc;
    }
}

// Contractions -lambda^T (dA/dtheta) psi = lambda^T (dF/dtheta) psi for the parameters of
// q-dependent channels (Eq. FE, F = sum_mu P_j g_(j,j') P_j'), per level kappa of the vibrational
// basis, with u^x_j = (P_j x_(d_j))(kappa) and g_(j,j') = F[f_j f_j'](E - E_kappa):
//   a_j : sum_j' g_(j,j') / (2 a_j) (u^lam_j u^psi_j' + u^lam_j' u^psi_j)  (dg_(j,j)/da_j = g_(j,j)/a_j)
//   b_j : sum_j' h_(j,j') / 2 (u^lam_j u^psi_j' + u^lam_j' u^psi_j),  h = dg/db = -F^(l+1)
//   c_t of P_j : (Q_t lam_(d_j)) W^psi_j + (Q_t psi_(d_j)) W^lam_j,  W^x_j = sum_j' g_(j,j') u^x_j'
// (Q_t the unit-coefficient term, symmetric).  part[s][blk][theta]; zero for other parameters.
template <int M>
__global__ void __launch_bounds__(TPB) k_adjoint_sand(DevModel md, const double* __restrict__ Etot,
                                                     const double2* __restrict__ lam, const double2* __restrict__ psi,
                                                     int ntheta, const GradParam* __restrict__ gp,
                                                     const DevEntry* __restrict__ pts, double* __restrict__ part) {
    __shared__ double red[TPB / 32];
    const int s = blockIdx.y, Nnu = md.Nnu;
    const int kap = blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = kap < Nnu;
    const double2* ls = lam + (long long)s * md.N;
    const double2* ps = psi + (long long)s * md.N;
    double2 ul[MAXCH], up[MAXCH];
    double eps = 0.0;
    int n[MAXM];
    if (on) {
        eps = Etot[s / md.nmu] - md.enu[kap];
        decode_nu<M>(md, kap, n);
        for (int j = 0; j < md.nsc; ++j) {
            double2 a = make_double2(0.0, 0.0), b = a;
            const long long od = (long long)md.sc_d[j] * Nnu;
            for (int k = md.sc_pbeg[j]; k < md.sc_pbeg[j + 1]; ++k) {
                const double cf = md.spc64[(long long)k * Nnu + kap];
                if (cf == 0.0) continue;
                const double2 xl = ls[od + kap + md.sp_lin[k]], xp = ps[od + kap + md.sp_lin[k]];
                a.x += cf * xl.x;
                a.y += cf * xl.y;
                b.x += cf * xp.x;
                b.y += cf * xp.y;
            }
            ul[j] = a;
            up[j] = b;
        }
    }
    auto pair_shift = [&](int p, int dl) {
        return vbk_level_shift_core(eps, md.pr_a[p], md.pr_b[p], md.pr_sb[p], md.pr_isb[p], md.pr_ib[p], md.pr_l[p] + dl);
    };
    for (int th = 0; th < ntheta; ++th) {
        const GradParam g = gp[th];
        double v = 0.0;
        if (on && g.j >= 0) {
            const int j = g.j;
            if (g.kind == 1 || g.kind == 2) {
                double2 acc = make_double2(0.0, 0.0);
                for (int j2 = 0; j2 < md.nsc; ++j2) {
                    const int p = md.sc_pair[j][j2];
                    if (p < 0) continue;
                    double2 G = g.kind == 1 ? pair_shift(p, 0) : pair_shift(p, 1);
                    const double sc = g.kind == 1 ? 0.5 / md.ch_a[g.c] : -0.5;
                    G = make_double2(sc * G.x, sc * G.y);
                    const double2 t = cadd<double>(cmul<double>(ul[j], up[j2]), cmul<double>(ul[j2], up[j]));
                    acc = cfma<double>(G, t, acc);
                }
                v = acc.x;
            } else if (g.kind == 3) {
                double2 wl = make_double2(0.0, 0.0), wp = wl;
                for (int j2 = 0; j2 < md.nsc; ++j2) {
                    const int p = md.sc_pair[j][j2];
                    if (p < 0) continue;
                    const double2 G = pair_shift(p, 0);
                    wl = cfma<double>(G, ul[j2], wl);
                    wp = cfma<double>(G, up[j2], wp);
                }
                double2 ql = make_double2(0.0, 0.0), qp = ql;
                const long long od = (long long)md.sc_d[j] * Nnu;
                for (int k = g.pb; k < g.pe; ++k) {
                    const DevEntry pt = pts[k];
                    double cf = 1.0;
                    bool ok = true;
#pragma unroll
                    for (int m = 0; m < M; ++m)
                        if (pt.col[m] >= 0) {
                            const int nn = n[m] + pt.delta[m];
                            ok = ok && nn >= 0 && nn < md.nb[m];
                            cf *= md.tab64[pt.col[m] + n[m]];
                        }
                    if (ok) {
                        const double2 xl = ls[od + kap + pt.lin], xp = ps[od + kap + pt.lin];
                        ql.x += cf * xl.x;
                        ql.y += cf * xl.y;
                        qp.x += cf * xp.x;
                        qp.y += cf * xp.y;
                    }
                }
                v = cadd<double>(cmul<double>(ql, wp), cmul<double>(qp, wl)).x;
            }
        }
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < TPB / 32; ++w) t += red[w];
            part[((long long)s * gridDim.x + blockIdx.x) * ntheta + th] = t;
        }
    }
}

// grad[theta] = sum_s sum_blk part[s][blk][theta] + sum_s sum_blk2 part2[s][blk2][theta]
//             + sum_s rhs_terms[s][theta]  (fixed order)
__global__ void k_grad_reduce(int nsys, int nblk, int nblk2, int ntheta, const double* __restrict__ part,
                              const double* __restrict__ part2, const double* __restrict__ rhs_terms,
                              double* __restrict__ grad) {
    const int th = blockIdx.x * blockDim.x + threadIdx.x;
    if (th >= ntheta) return;
    double acc = 0.0;
    for (int s = 0; s < nsys; ++s) {
        for (int b = 0; b < nblk; ++b) acc += part[((long long)s * nblk + b) * ntheta + th];
        for (int b = 0; b < nblk2; ++b) acc += part2[((long long)s * nblk2 + b) * ntheta + th];
        acc += rhs_terms[(long long)s * ntheta + th];
    }
    grad[th] = acc;
}

// rows idx[k] of src into row k of dst (gather) or row k of src into rows idx[k] of dst (scatter)
__global__ void k_move_rows(int n, int N, const int* __restrict__ idx, const double2* __restrict__ src,
                            double2* __restrict__ dst, int scatter) {
    const int k = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || i >= N) return;
    const long long a = (long long)idx[k] * N + i, c = (long long)k * N + i;
    if (scatter)
        dst[a] = src[c];
    else
        dst[c] = src[a];
}

// A VBK_MIXED COCG solve whose FP32 inner iterations stop helping a system (the FP64 residual of a
// refinement step falls by less than 10%, or a non-finite value or a breakdown appears) solves
// that system again in FP64 from x = 0; its statistics then add both runs.
int solve_job_with_fallback(vbk_model* m, const SolveJob& job, const vbk_opts& o, vbk_stats* stats, cudaStream_t st) {
    std::vector<vbk_stats> own;
    vbk_stats* sv = stats;
    if (!sv) {
        own.resize(job.nsys);
        sv = own.data();
    }
    int rc = vbk_solve_job(m, job, o, sv, st);
    if (o.precision != VBK_MIXED || o.method != VBK_COCG || rc != VBK_ERR_NOT_CONVERGED) return rc;
    std::vector<int> redo;
    for (int s = 0; s < job.nsys; ++s)
        if (sv[s].status == VBK_SYS_STALLED || sv[s].status == VBK_SYS_NAN || sv[s].status == VBK_SYS_BREAKDOWN)
            redo.push_back(s);
    if (redo.empty()) return rc;
    const std::vector<KTimer> timers = m->timers;
    const long long launches = m->launches;
    const int nf = (int)redo.size(), N = m->N;
    const size_t rows = (size_t)nf * N * sizeof(double2), ib = ((size_t)nf * sizeof(int) + 255) & ~size_t(255);
    DevBuf buf;
    buf.st = st;
    VBK_CUDA(vbk_alloc(m, &buf.p, 2 * rows + ib, st));
    double2* bsub = (double2*)buf.p;
    double2* xsub = (double2*)((char*)buf.p + rows);
    int* didx = (int*)((char*)buf.p + 2 * rows);
    VBK_CUDA(cudaMemcpyAsync(didx, redo.data(), nf * sizeof(int), cudaMemcpyHostToDevice, st));
    const dim3 g(cdiv_u(N, TPB), (unsigned)nf);
    k_move_rows<<<g, TPB, 0, st>>>(nf, N, didx, job.b64, bsub, 0);
    VBK_CUDA(cudaGetLastError());
    SolveJob sub;
    sub.nsys = nf;
    sub.nE = job.nE;
    sub.E = job.E;
    for (int s : redo) sub.sys_e.push_back(job.sys_e[s]);
    sub.b64 = bsub;
    sub.x64 = xsub;
    vbk_opts o64 = o;
    o64.precision = VBK_FP64;
    std::vector<vbk_stats> s2(nf);
    const int rc2 = vbk_solve_job(m, sub, o64, s2.data(), st);
    if (rc2 != VBK_OK && rc2 != VBK_ERR_NOT_CONVERGED) return rc2;
    k_move_rows<<<g, TPB, 0, st>>>(nf, N, didx, xsub, job.x64, 1);
    VBK_CUDA(cudaGetLastError());
    VBK_CUDA(cudaStreamSynchronize(st));  // `redo` must outlive its copy
    bool ok = true;
    for (int k = 0; k < nf; ++k) {
        vbk_stats& S = sv[redo[k]];
        S.status = s2[k].status;
        S.iterations += s2[k].iterations;
        S.refinements += s2[k].refinements;
        S.rel_residual = s2[k].rel_residual;
    }
    for (int s = 0; s < job.nsys; ++s) ok = ok && (sv[s].status == VBK_SYS_CONVERGED || sv[s].status == VBK_SYS_ZERO_RHS);
    // kernel bookkeeping of both runs
    std::vector<KTimer> merged = timers;
    for (const KTimer& t : m->timers) {
        bool found = false;
        for (KTimer& u : merged)
            if (u.name == t.name) {
                u.launches += t.launches;
                u.ms += t.ms;
                found = true;
            }
        if (!found) merged.push_back(t);
    }
    m->timers = merged;
    m->launches += launches + 2;
    return ok ? VBK_OK : VBK_ERR_NOT_CONVERGED;
}

}  // namespace

// =============================================================================== C ABI
extern "C" {

void vbk_default_opts(vbk_opts* o) {
    if (!o) return;
    o->method = VBK_GMRES;
    o->precision = VBK_MIXED;
    o->precond_span = 0;
    o->restart = 64;
    o->max_iter = 20000;
    o->max_refine = 40;
    o->tol = 1e-8;
    o->inner_tol = 1e-5;
    o->check_every = 8;
    o->timing = 0;
    o->autotune = 1;
    o->resident = 1;
    o->inner_max_iter = 2000;
    o->matvec_variant = -1;
}

int vbk_build_model(const vbk_model_desc* desc, vbk_model** out) {
    g_last_error.clear();
    if (!out) return invalid("output handle pointer is NULL");
    *out = nullptr;
    if (int rc = validate_desc(desc)) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        g_last_error = "no CUDA device visible";
        return VBK_ERR_NO_DEVICE;
    }
    vbk_model* m = new (std::nothrow) vbk_model();
    if (!m) return VBK_ERR_OOM;
    cudaGetDevice(&m->device);
    {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = m->device;
        if (cudaMemPoolCreate(&m->pool, &props) == cudaSuccess) {
            unsigned long long thr = ~0ULL;
            cudaMemPoolSetAttribute(m->pool, cudaMemPoolAttrReleaseThreshold, &thr);
        } else {
            cudaGetLastError();
            m->pool = nullptr;  // fall back to the device's default pool
        }
    }
    int rc = build(desc, m);
    if (rc) {
        vbk_free_model(m);
        return rc;
    }
    *out = m;
    return VBK_OK;
}

void vbk_free_model(vbk_model* m) {
    if (!m) return;
    if (m->dev_mem) cudaFree(m->dev_mem);
    if (m->dev_mem2) cudaFree(m->dev_mem2);
    if (m->dev_mem3) cudaFree(m->dev_mem3);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    if (m->pool) {
        cudaDeviceSynchronize();  // outstanding frees of this model's calls complete before the pool goes
        cudaMemPoolDestroy(m->pool);
    }
    if (m->hpin) cudaFreeHost(m->hpin);
    delete m;
}

int vbk_model_size(const vbk_model* m, int* n_unknowns, int* n_partial_waves) {
    if (int rc = check_model(m)) return rc;
    if (n_unknowns) *n_unknowns = m->N;
    if (n_partial_waves) *n_partial_waves = m->nmu;
    return VBK_OK;
}

static int check_opts(const vbk_opts* o) {
    if (!o) return invalid("options are NULL");
    if (o->method != VBK_GMRES && o->method != VBK_COCG) return invalid("unknown Krylov method");
    if (o->precision != VBK_FP64 && o->precision != VBK_MIXED) return invalid("unknown precision");
    if (o->restart < 1 || o->restart > 256) return invalid("restart must be in 1..256");
    if (o->max_iter < 1 || o->max_refine < 1) return invalid("max_iter and max_refine must be >= 1");
    if (!(o->tol > 0.0) || !(o->tol < 1.0)) return invalid("tol must be in (0, 1)");
    if (!(o->inner_tol > 0.0) || !(o->inner_tol < 1.0)) return invalid("inner_tol must be in (0, 1)");
    if (o->check_every < 1) return invalid("check_every must be >= 1");
    if (o->precond_span < -1) return invalid("precond_span must be -1 or a span mask");
    if (o->inner_max_iter < 0) return invalid("inner_max_iter must be >= 0");
    if (o->resident < 0 || o->resident > 3) return invalid("resident must be 0, 1, 2 or 3");
    if (o->matvec_variant < -1 || o->matvec_variant >= VBK_MATVEC_NVARIANTS)
        return invalid("matvec_variant must be -1 or a variant index");
    return VBK_OK;
}

// Shared set-up of solve / adjoint: energies, distinct-energy map, flat initial indices.
static int make_systems(vbk_model* m, int n_eps, const double* eps, int n_vi, const int* vi, SolveJob* job,
                        std::vector<double>* Etot, std::vector<int>* vflat, std::vector<double>* Evi) {
    if (n_eps < 1 || n_vi < 1 || !eps || !vi) return invalid("n_eps, n_vi, eps_i and vi must be given");
    if ((long long)n_eps * n_vi * m->nmu > 65535) return invalid("at most 65535 systems (energies x initial states x partial waves) per call");
    for (int e = 0; e < n_eps; ++e)
        if (!(eps[e] > 0.0) || !std::isfinite(eps[e])) return invalid("incident energies must be positive and finite");
    vflat->resize(n_vi);
    Evi->resize(n_vi);
    for (int i = 0; i < n_vi; ++i) {
        if (int rc = flat_index(m, vi + (long long)i * m->M, &(*vflat)[i])) return rc;
        (*Evi)[i] = level_energy(m, vi + (long long)i * m->M);
    }
    Etot->resize((size_t)n_eps * n_vi);
    std::map<double, int> idx;
    job->E.clear();
    job->sys_e.clear();
    for (int e = 0; e < n_eps; ++e)
        for (int i = 0; i < n_vi; ++i) {
            const double E = eps[e] + (*Evi)[i];
            (*Etot)[(size_t)e * n_vi + i] = E;
            auto it = idx.find(E);
            int k;
            if (it == idx.end()) {
                k = (int)job->E.size();
                idx[E] = k;
                job->E.push_back(E);
            } else {
                k = it->second;
            }
            for (int mu = 0; mu < m->nmu; ++mu) job->sys_e.push_back(k);
        }
    job->nE = (int)job->E.size();
    job->nsys = (int)job->sys_e.size();
    return VBK_OK;
}

int vbk_solve(vbk_model* m, int n_eps, const double* eps_i, int n_vi, const int* vi, const vbk_opts* opts, void* psi_dev,
              vbk_stats* stats, void* stream) {
    g_last_error.clear();
    if (int rc = check_model(m)) return rc;
    if (int rc = check_opts(opts)) return rc;
    if (!psi_dev) return invalid("psi_dev is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    SolveJob job;
    std::vector<double> Etot, Evi;
    std::vector<int> vflat;
    if (int rc = make_systems(m, n_eps, eps_i, n_vi, vi, &job, &Etot, &vflat, &Evi)) return rc;
    const size_t N = m->N;
    DevBuf b;
    b.st = st;
    const size_t bbytes = (size_t)job.nsys * N * sizeof(double2);
    const size_t o_vf = (((size_t)n_eps * sizeof(double) + 255) & ~size_t(255));
    const size_t o_bn = o_vf + (((size_t)n_vi * sizeof(int) + 255) & ~size_t(255));
    const size_t extra = o_bn + (size_t)job.nsys * sizeof(double);
    VBK_CUDA(vbk_alloc(m, &b.p, bbytes + extra, st));
    double2* b64 = (double2*)b.p;
    double* deps = (double*)((char*)b.p + bbytes);
    int* dvf = (int*)((char*)deps + o_vf);
    double* bn2 = (double*)((char*)deps + o_bn);
    VBK_CUDA(cudaMemsetAsync(b64, 0, bbytes, st));
    VBK_CUDA(cudaMemcpyAsync(deps, eps_i, n_eps * sizeof(double), cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(dvf, vflat.data(), n_vi * sizeof(int), cudaMemcpyHostToDevice, st));
    k_build_rhs<<<cdiv_u(job.nsys, 128), 128, 0, st>>>(m->dm, job.nsys, n_vi, deps, dvf, b64, bn2);
    VBK_CUDA(cudaGetLastError());
    job.b64 = b64;
    job.bnorm2 = bn2;
    job.x64 = (double2*)psi_dev;
    int rc = solve_job_with_fallback(m, job, *opts, stats, st);
    m->launches += 1;  // k_build_rhs
    return rc;
}

int vbk_cross_sections(vbk_model* m, int n_eps, const double* eps_i, int n_vi, const int* vi, const void* psi_dev, int n_vf,
                       const int* vf, double* sigma_dev, void* t_dev, void* stream) {
    g_last_error.clear();
    if (int rc = check_model(m)) return rc;
    if (!psi_dev || !sigma_dev) return invalid("psi_dev and sigma_dev must be given");
    if (n_vf < 1 || !vf) return invalid("final states missing");
    cudaStream_t st = (cudaStream_t)stream;
    SolveJob job;
    std::vector<double> Etot, Evi;
    std::vector<int> vflat;
    if (int rc = make_systems(m, n_eps, eps_i, n_vi, vi, &job, &Etot, &vflat, &Evi)) return rc;
    std::vector<int> ff(n_vf);
    std::vector<double> Ef(n_vf);
    for (int f = 0; f < n_vf; ++f) {
        if (int rc = flat_index(m, vf + (long long)f * m->M, &ff[f])) return rc;
        Ef[f] = level_energy(m, vf + (long long)f * m->M);
    }
    DevBuf b;
    b.st = st;
    const size_t s1 = ((size_t)n_eps * 8 + 255) & ~size_t(255), s2 = (Etot.size() * 8 + 255) & ~size_t(255),
                 s3 = ((size_t)n_vf * 4 + 255) & ~size_t(255), s4 = ((size_t)n_vf * 8 + 255) & ~size_t(255);
    VBK_CUDA(vbk_alloc(m, &b.p, s1 + s2 + s3 + s4, st));
    char* p = (char*)b.p;
    VBK_CUDA(cudaMemcpyAsync(p, eps_i, n_eps * 8, cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(p + s1, Etot.data(), Etot.size() * 8, cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(p + s1 + s2, ff.data(), n_vf * 4, cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(p + s1 + s2 + s3, Ef.data(), n_vf * 8, cudaMemcpyHostToDevice, st));
    const long long nt = (long long)n_eps * n_vi * n_vf;
    k_sigma<<<cdiv_u(nt, 128), 128, 0, st>>>(m->dm, n_eps, n_vi, n_vf, (const double*)p, (const double*)(p + s1),
                                             (const double2*)psi_dev, (const int*)(p + s1 + s2), (const double*)(p + s1 + s2 + s3),
                                             sigma_dev, (double2*)t_dev);
    VBK_CUDA(cudaGetLastError());
    return VBK_OK;
}

int vbk_eels(vbk_model* m, int n_eps, int n_vi, const int* vi, int n_vf, const int* vf, const double* sigma_dev, int n_de,
             const double* de, double fwhm, double* S_dev, void* stream) {
    g_last_error.clear();
    if (int rc = check_model(m)) return rc;
    if (n_eps < 1 || n_vi < 1 || n_vf < 1 || n_de < 1 || !vi || !vf || !de || !sigma_dev || !S_dev)
        return invalid("eels: sizes and buffers must be given");
    if (!(fwhm > 0.0)) return invalid("fwhm must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> Ef(n_vf), Ei(n_vi);
    for (int f = 0; f < n_vf; ++f) {
        int tmp;
        if (int rc = flat_index(m, vf + (long long)f * m->M, &tmp)) return rc;
        Ef[f] = level_energy(m, vf + (long long)f * m->M);
    }
    for (int i = 0; i < n_vi; ++i) {
        int tmp;
        if (int rc = flat_index(m, vi + (long long)i * m->M, &tmp)) return rc;
        Ei[i] = level_energy(m, vi + (long long)i * m->M);
    }
    DevBuf b;
    b.st = st;
    const size_t s1 = ((size_t)n_de * 8 + 255) & ~size_t(255), s2 = ((size_t)n_vf * 8 + 255) & ~size_t(255),
                 s3 = ((size_t)n_vi * 8 + 255) & ~size_t(255);
    VBK_CUDA(vbk_alloc(m, &b.p, s1 + s2 + s3, st));
    char* p = (char*)b.p;
    VBK_CUDA(cudaMemcpyAsync(p, de, n_de * 8, cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(p + s1, Ef.data(), n_vf * 8, cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(p + s1 + s2, Ei.data(), n_vi * 8, cudaMemcpyHostToDevice, st));
    const double sdev = fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    const long long nt = (long long)n_eps * n_vi * n_de;
    k_eels<<<cdiv_u(nt, 128), 128, 0, st>>>(n_eps, n_vi, n_vf, n_de, sigma_dev, (const double*)p, (const double*)(p + s1),
                                            (const double*)(p + s1 + s2), sdev, S_dev);
    VBK_CUDA(cudaGetLastError());
    return VBK_OK;
}

int vbk_solve_adjoint(vbk_model* m, int n_eps, const double* eps_i, int n_vi, const int* vi, const vbk_opts* opts,
                      const void* psi_dev, int n_vf, const int* vf, const double* dL_dsigma_dev, int n_theta,
                      const int* theta_ids, double* grad, vbk_stats* stats, void* stream) {
    g_last_error.clear();
    if (int rc = check_model(m)) return rc;
    if (int rc = check_opts(opts)) return rc;
    if (!psi_dev || !dL_dsigma_dev || !grad || !theta_ids) return invalid("adjoint: buffers must be given");
    if (n_vf < 1 || !vf || n_theta < 1 || n_theta > 4096) return invalid("adjoint: n_vf >= 1 and 1 <= n_theta <= 4096");
    cudaStream_t st = (cudaStream_t)stream;
    SolveJob job;
    std::vector<double> Etot, Evi;
    std::vector<int> vflat;
    if (int rc = make_systems(m, n_eps, eps_i, n_vi, vi, &job, &Etot, &vflat, &Evi)) return rc;
    std::vector<int> ff(n_vf);
    std::vector<double> Ef(n_vf);
    for (int f = 0; f < n_vf; ++f) {
        if (int rc = flat_index(m, vf + (long long)f * m->M, &ff[f])) return rc;
        Ef[f] = level_energy(m, vf + (long long)f * m->M);
    }
    // parameter descriptors and the point lists of the term parameters
    const int nterm = (int)m->terms.size();
    std::vector<GradParam> gps(n_theta);
    std::vector<DevEntry> pts;
    std::vector<int> ptd;
    const int nch = (int)m->chans.size(), nct = (int)m->cterms.size();
    auto sand_index = [&](int c) {
        for (int j = 0; j < m->dm.nsc; ++j)
            if (m->dm.sc_ch[j] == c) return j;
        return -1;
    };
    for (int k = 0; k < n_theta; ++k) {
        const int id = theta_ids[k];
        if (id < 0 || id >= nterm + 2 * nch + nct) return invalid("theta id out of range");
        GradParam g{0, 0, 0, 0, -1};
        if (id >= nterm + 2 * nch) {
            // coefficient of coupling term t: the unit-coefficient points of its polynomial term
            const vbk_cterm& t = m->cterms[id - nterm - 2 * nch];
            g.kind = 3;
            g.c = t.channel;
            g.j = sand_index(t.channel);
            g.pb = (int)pts.size();
            int cnt[MAXM], o[MAXM];
            long long ncomb = 1;
            for (int q = 0; q < m->M; ++q) {
                cnt[q] = t.pow[q] + 1;
                ncomb *= cnt[q];
            }
            for (long long cb = 0; cb < ncomb; ++cb) {
                long long rem = cb;
                for (int q = m->M - 1; q >= 0; --q) {
                    o[q] = (int)(rem % cnt[q]);
                    rem /= cnt[q];
                }
                DevEntry e{};
                e.coef = 1.0;
                e.dp = m->chans[t.channel].d;
                for (int q = 0; q < MAXM; ++q) {
                    e.col[q] = -1;
                    e.delta[q] = 0;
                }
                for (int q = 0; q < m->M; ++q) {
                    if (!t.pow[q]) continue;
                    e.delta[q] = -t.pow[q] + 2 * o[q];
                    e.col[q] = m->colbase[q][t.pow[q]] + o[q] * m->nb[q];
                    e.lin += e.delta[q] * m->stride[q];
                }
                pts.push_back(e);
                ptd.push_back(-1);  // not a U point: never matched by the element-wise contraction
            }
            g.pe = (int)pts.size();
            gps[k] = g;
            continue;
        }
        if (id < nterm) {
            g.kind = 0;
            g.pb = (int)pts.size();
            for (const auto* lst : {&m->offd, &m->diagp})
                for (const auto& he : *lst)
                    if (he.term == id) {
                        DevEntry e = he.e;
                        e.coef = he.w;  // derivative of the point's coefficient in the term's
                        pts.push_back(e);
                        ptd.push_back(he.d);
                    }
            g.pe = (int)pts.size();
        } else {
            g.kind = 1 + (id - nterm) % 2;
            g.c = (id - nterm) / 2;
            if (g.kind == 1 && !(m->chans[g.c].a > 0.0)) return invalid("gradient in a needs a > 0");
            g.j = m->dm.ch_sw[g.c] ? sand_index(g.c) : -1;
        }
        gps[k] = g;
    }
    if (pts.empty()) {
        pts.push_back(DevEntry{});
        ptd.push_back(-1);
    }
    const size_t N = m->N;
    const long long nsys = job.nsys;
    const int nblk = (int)cdiv_u(N, TPB);
    const int nblk2 = m->dm.nsc ? (int)cdiv_u(m->Nnu, TPB) : 0;  // sandwich contractions per level
    const int nmu = m->nmu;
    const size_t nT = (size_t)n_eps * n_vi * nmu * n_vf * nmu;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t off[17];
    size_t tot = 0;
    size_t sizes[] = {al(nsys * N * sizeof(double2)),                      // 0 g (adjoint rhs)
                      al(nsys * N * sizeof(double2)),                      // 1 lambda
                      al(nT * sizeof(double2)),                            // 2 T
                      al(nT * sizeof(double2)),                            // 3 W
                      al((size_t)n_eps * 8), al(Etot.size() * 8),          // 4 eps, 5 Etot
                      al((size_t)n_vf * 4), al((size_t)n_vf * 8),          // 6 vf flat, 7 E_vf
                      al((size_t)n_vi * 4), al((size_t)n_vi * 8),          // 8 vi flat, 9 E_vi
                      al(gps.size() * sizeof(GradParam)),                  // 10
                      al(pts.size() * sizeof(DevEntry)), al(ptd.size() * 4),  // 11, 12
                      al(nsys * (size_t)nblk * n_theta * 8),               // 13 partials
                      al(nsys * (size_t)n_theta * 8),                      // 14 rhs terms
                      al((size_t)n_theta * 8),                             // 15 grad (device)
                      al(nsys * (size_t)nblk2 * n_theta * 8 + 8)};         // 16 sandwich partials
    for (int k = 0; k < 17; ++k) {
        off[k] = tot;
        tot += sizes[k];
    }
    DevBuf b;
    b.st = st;
    VBK_CUDA(vbk_alloc(m, &b.p, tot, st));
    char* p = (char*)b.p;
    auto P = [&](int k) { return p + off[k]; };
    VBK_CUDA(cudaMemsetAsync(P(0), 0, sizes[0], st));
    VBK_CUDA(cudaMemcpyAsync(P(4), eps_i, n_eps * 8, cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(P(5), Etot.data(), Etot.size() * 8, cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(P(6), ff.data(), n_vf * 4, cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(P(7), Ef.data(), n_vf * 8, cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(P(8), vflat.data(), n_vi * 4, cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(P(9), Evi.data(), n_vi * 8, cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(P(10), gps.data(), gps.size() * sizeof(GradParam), cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(P(11), pts.data(), pts.size() * sizeof(DevEntry), cudaMemcpyHostToDevice, st));
    VBK_CUDA(cudaMemcpyAsync(P(12), ptd.data(), ptd.size() * 4, cudaMemcpyHostToDevice, st));
    // T from the forward solutions, adjoint right-hand sides
    const long long nt = (long long)n_eps * n_vi * n_vf;
    std::vector<double> sig_dummy;  // sigma itself is not needed here
    double* dsig = nullptr;
    VBK_CUDA(vbk_alloc(m, (void**)&dsig, std::max<long long>(1, nt) * sizeof(double), st));
    k_sigma<<<cdiv_u(nt, 128), 128, 0, st>>>(m->dm, n_eps, n_vi, n_vf, (const double*)P(4), (const double*)P(5),
                                             (const double2*)psi_dev, (const int*)P(6), (const double*)P(7), dsig,
                                             (double2*)P(2));
    k_adjoint_rhs<<<cdiv_u(nsys, 128), 128, 0, st>>>(m->dm, n_eps, n_vi, n_vf, (const double*)P(4), (const double*)P(5),
                                                     (const double2*)P(2), dL_dsigma_dev, (const int*)P(6),
                                                     (const double*)P(7), (double2*)P(0), (double2*)P(3));
    cudaFreeAsync(dsig, st);
    VBK_CUDA(cudaGetLastError());
    // lambda = A^-1 g  (A = A^T: the forward operator serves as its own transpose)
    job.b64 = (const double2*)P(0);
    job.x64 = (double2*)P(1);
    int rc = solve_job_with_fallback(m, job, *opts, stats, st);
    if (rc != VBK_OK && rc != VBK_ERR_NOT_CONVERGED) return rc;
    const long long extra_launches = nblk2 ? 6 : 5;
    // contractions
    const dim3 gc(nblk, (unsigned)nsys);
    switch (m->M) {
        case 1: k_adjoint_contract<1><<<gc, TPB, 0, st>>>(m->dm, (int)nsys, n_vi, (const double*)P(5), (const double2*)P(1), (const double2*)psi_dev, n_theta, (const GradParam*)P(10), (const int*)P(12), (const DevEntry*)P(11), (double*)P(13)); break;
        case 2: k_adjoint_contract<2><<<gc, TPB, 0, st>>>(m->dm, (int)nsys, n_vi, (const double*)P(5), (const double2*)P(1), (const double2*)psi_dev, n_theta, (const GradParam*)P(10), (const int*)P(12), (const DevEntry*)P(11), (double*)P(13)); break;
        case 3: k_adjoint_contract<3><<<gc, TPB, 0, st>>>(m->dm, (int)nsys, n_vi, (const double*)P(5), (const double2*)P(1), (const double2*)psi_dev, n_theta, (const GradParam*)P(10), (const int*)P(12), (const DevEntry*)P(11), (double*)P(13)); break;
        default: k_adjoint_contract<4><<<gc, TPB, 0, st>>>(m->dm, (int)nsys, n_vi, (const double*)P(5), (const double2*)P(1), (const double2*)psi_dev, n_theta, (const GradParam*)P(10), (const int*)P(12), (const DevEntry*)P(11), (double*)P(13)); break;
    }
    if (nblk2) {
        const dim3 gs(nblk2, (unsigned)nsys);
        switch (m->M) {
            case 1: k_adjoint_sand<1><<<gs, TPB, 0, st>>>(m->dm, (const double*)P(5), (const double2*)P(1), (const double2*)psi_dev, n_theta, (const GradParam*)P(10), (const DevEntry*)P(11), (double*)P(16)); break;
            case 2: k_adjoint_sand<2><<<gs, TPB, 0, st>>>(m->dm, (const double*)P(5), (const double2*)P(1), (const double2*)psi_dev, n_theta, (const GradParam*)P(10), (const DevEntry*)P(11), (double*)P(16)); break;
            case 3: k_adjoint_sand<3><<<gs, TPB, 0, st>>>(m->dm, (const double*)P(5), (const double2*)P(1), (const double2*)psi_dev, n_theta, (const GradParam*)P(10), (const DevEntry*)P(11), (double*)P(16)); break;
            default: k_adjoint_sand<4><<<gs, TPB, 0, st>>>(m->dm, (const double*)P(5), (const double2*)P(1), (const double2*)psi_dev, n_theta, (const GradParam*)P(10), (const DevEntry*)P(11), (double*)P(16)); break;
        }
    }
    k_adjoint_rhs_terms<<<cdiv_u(nsys, 128), 128, 0, st>>>(m->dm, n_eps, n_vi, n_vf, (const double*)P(4), (const double*)P(5),
                                                           (const int*)P(8), (const double*)P(9), (const int*)P(6),
                                                           (const double*)P(7), (const double2*)P(3), (const double2*)P(1),
                                                           (const double2*)psi_dev, n_theta, (const GradParam*)P(10),
                                                           (const DevEntry*)P(11), (double*)P(14));
    k_grad_reduce<<<cdiv_u(n_theta, 64), 64, 0, st>>>((int)nsys, nblk, nblk2, n_theta, (const double*)P(13),
                                                      (const double*)P(16), (const double*)P(14), (double*)P(15));
    VBK_CUDA(cudaGetLastError());
    VBK_CUDA(cudaMemcpyAsync(grad, P(15), n_theta * 8, cudaMemcpyDeviceToHost, st));
    VBK_CUDA(cudaStreamSynchronize(st));
    m->launches += extra_launches;
    return rc;
}

int vbk_matvec(vbk_model* m, int n_E, const double* E, int n_vec, const void* x_dev, void* y_dev, int precision,
               int variant, void* stream) {
    g_last_error.clear();
    if (int rc = check_model(m)) return rc;
    if (n_E < 1 || n_vec < 1 || !E || !x_dev || !y_dev) return invalid("matvec: sizes and buffers must be given");
    if (precision != VBK_FP64 && precision != VBK_MIXED) return invalid("unknown precision");
    for (int k = 0; k < n_E; ++k)
        if (!std::isfinite(E[k])) return invalid("energies must be finite");
    if (variant < -1) return invalid("matvec variant must be -1 or a variant index");
    return vbk_operator_run(m, 0, n_E, E, n_vec, 0, (const double2*)x_dev, (double2*)y_dev, precision,
                            (cudaStream_t)stream, variant);
}

int vbk_precond_apply(vbk_model* m, int n_E, const double* E, int n_vec, int precond_span, const void* r_dev, void* z_dev,
                      int precision, void* stream) {
    g_last_error.clear();
    if (int rc = check_model(m)) return rc;
    if (n_E < 1 || n_vec < 1 || !E || !r_dev || !z_dev) return invalid("precond: sizes and buffers must be given");
    if (precision != VBK_FP64 && precision != VBK_MIXED) return invalid("unknown precision");
    if (precond_span < -1 || precond_span >= (2 << m->M)) return invalid("precond_span out of range");
    for (int k = 0; k < n_E; ++k)
        if (!std::isfinite(E[k])) return invalid("energies must be finite");
    return vbk_operator_run(m, 1, n_E, E, n_vec, precond_span, (const double2*)r_dev, (double2*)z_dev, precision,
                            (cudaStream_t)stream);
}

int vbk_level_shift_df(double eps, double a, double b, int l, double* re, double* im) {
    g_last_error.clear();
    if (!re || !im) return invalid("level shift: output pointers must be given");
    if (!std::isfinite(eps) || !(a >= 0.0) || !std::isfinite(a) || !(b > 0.0) || !std::isfinite(b) || l < 0 || l > 20)
        return invalid("level shift: eps finite, a >= 0, b > 0, 0 <= l <= 20");
    static std::vector<float2> dws, erx, tay;
    static std::once_flag once;
    std::call_once(once, [] { vbk_df_tables(&dws, &erx, &tay); });
    const DfLevelShift T{dws.data(), erx.data(), tay.data(), VBK_ERFCX_NINT};
    const double cv[5] = {a, b, std::sqrt(b), 1.0 / std::sqrt(b), 1.0 / b};
    float2 c[5];
    for (int q = 0; q < 5; ++q) {
        const dflt v = dd_from(cv[q]);
        c[q] = make_float2(v.h, v.l);
    }
    dflt fr, fi;
    dd_level_shift(dd_from(eps), c, l, T, &fr, &fi);
    *re = dd_to_double(fr);
    *im = dd_to_double(fi);
    return VBK_OK;
}

int vbk_set_op_timing(vbk_model* m, int on) {
    g_last_error.clear();
    if (int rc = check_model(m)) return rc;
    m->op_timing = on ? 1 : 0;
    return VBK_OK;
}

int vbk_kernel_timings(const vbk_model* m, int cap, const char** names, int* launches, double* total_ms) {
    if (!m) return 0;
    const int n = (int)m->timers.size();
    for (int k = 0; k < n && k < cap; ++k) {
        if (names) names[k] = m->timers[k].name.c_str();
        if (launches) launches[k] = (int)m->timers[k].launches;
        if (total_ms) total_ms[k] = m->timers[k].ms;
    }
    return n;
}

long long vbk_last_launch_count(const vbk_model* m) { return m ? m->launches : 0; }

int vbk_debug_stream_delay(int ms) {
    vbk_set_error("");
    const int rc = vbk_debug_stream_delay_impl(ms);
    if (rc) vbk_set_error("delay must be in 0 .. 10000 ms");
    return rc;
}

int vbk_matvec_variant(const vbk_model* m, int precision) {
    if (!m) return -1;
    return m->mv_variant[precision == VBK_MIXED ? 0 : 1];
}

const char* vbk_status_str(int code) {
    switch (code) {
        case VBK_OK: return "ok";
        case VBK_ERR_INVALID_ARG: return "invalid argument";
        case VBK_ERR_OOM: return "out of memory";
        case VBK_ERR_CUDA: return "CUDA error";
        case VBK_ERR_NOT_CONVERGED: return "not converged";
        case VBK_ERR_UNSUPPORTED: return "unsupported";
        case VBK_ERR_NO_DEVICE: return "no CUDA device";
    }
    return "unknown status";
}

const char* vbk_sys_status_str(int status) {
    switch (status) {
        case VBK_SYS_CONVERGED: return "converged";
        case VBK_SYS_MAX_ITER: return "iteration limit";
        case VBK_SYS_BREAKDOWN: return "breakdown";
        case VBK_SYS_NAN: return "non-finite value";
        case VBK_SYS_PIVOT: return "zero pivot in preconditioner";
        case VBK_SYS_ZERO_RHS: return "zero right-hand side";
    }
    return "unknown system status";
}

const char* vbk_last_error(void) { return g_last_error.c_str(); }

int vbk_level_shift(double eps, double a, double b, int l, double* re, double* im) {
    if (!re || !im) return invalid("output pointers are NULL");
    if (!std::isfinite(eps) || !(a >= 0.0) || !(b > 0.0) || l < 0 || l > 20) return invalid("level shift parameters out of range");
    const double2 F = vbk_level_shift_eval(eps, a, b, l);
    *re = F.x;
    *im = F.y;
    return VBK_OK;
}

}  // extern "C"

// ------------------------------------------------------------------- block plans (host)
int vbk_make_block_plan(const vbk_model* m, int span, BlockPlan* bp) {
    if (span <= 0 || span >= (2 << m->M)) {
        g_last_error = "block preconditioner span out of range";
        return VBK_ERR_INVALID_ARG;
    }
    bp->span = span;
    const bool sd = span & 1;
    long long L = sd ? m->ns : 1;
    long long cstr[MAXM] = {0};
    long long acc = sd ? m->ns : 1;
    for (int k = m->M - 1; k >= 0; --k)
        if (span & (2 << k)) {
            cstr[k] = acc;
            acc *= m->nb[k];
        }
    L = acc;
    bp->L = (int)L;
    bp->nblk = (int)(m->N / L);
    bp->ent_dc.assign(m->offd.size(), 0);
    int p = 0;
    for (size_t k = 0; k < m->offd.size(); ++k) {
        const HostEntry& h = m->offd[k];
        bool in = sd || h.e.dp == h.d;
        long long dc = sd ? (h.e.dp - h.d) : 0;
        for (int mm = 0; mm < m->M && in; ++mm) {
            if (span & (2 << mm))
                dc += (long long)h.e.delta[mm] * cstr[mm];
            else if (h.e.delta[mm] != 0)
                in = false;
        }
        if (!in || dc == 0) continue;
        bp->ent_dc[k] = (int)dc;
        p = std::max<int>(p, (int)std::llabs(dc));
    }
    // entries of the sandwich operator (q-dependent couplings) that fall inside a block
    bp->sw_combo.clear();
    const DevModel& dm = m->dm;
    for (int j = 0; j < dm.nsc; ++j)
        for (int j2 = 0; j2 < dm.nsc; ++j2) {
            const int pr = dm.sc_pair[j][j2];
            if (pr < 0) continue;
            for (int k = dm.sc_pbeg[j]; k < dm.sc_pbeg[j + 1]; ++k)
                for (int k2 = dm.sc_pbeg[j2]; k2 < dm.sc_pbeg[j2 + 1]; ++k2) {
                    const int dd = dm.sc_d[j2] - dm.sc_d[j];
                    bool in = sd || dd == 0;
                    long long dc = sd ? dd : 0;
                    for (int mm = 0; mm < m->M && in; ++mm) {
                        const int delta = m->sp_delta[k][mm] + m->sp_delta[k2][mm];
                        if (span & (2 << mm))
                            dc += (long long)delta * cstr[mm];
                        else if (delta != 0)
                            in = false;
                    }
                    if (!in || dc == 0) continue;  // dc = 0: on the diagonal (in the diagonal tables)
                    bp->sw_combo.insert(bp->sw_combo.end(), {dm.sc_d[j], k, k2, pr, (int)dc});
                    p = std::max<int>(p, (int)std::llabs(dc));
                }
        }
    if (p > PWMAX) {
        g_last_error = "block preconditioner bandwidth " + std::to_string(p) + " exceeds the supported " + std::to_string(PWMAX);
        return VBK_ERR_UNSUPPORTED;
    }
    bp->p = p;
    bp->wide = p > PMAX;
    if (bp->wide) {
        bp->S = 4 * ((p + 7) / 8);  // levels of S >= p / 2 chain positions: block pentadiagonal
        bp->K = (bp->L + bp->S - 1) / bp->S;
        if (bp->nblk > 65535) {
            g_last_error = "wide-band block preconditioner with more than 65535 blocks";
            return VBK_ERR_UNSUPPORTED;
        }
    }
    return VBK_OK;
}
