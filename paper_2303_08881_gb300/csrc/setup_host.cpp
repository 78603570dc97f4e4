// setup_host.cpp -- host half of ilu_setup: validation, interior/interface classification,
// interior-first permutation, local blocks in Q order, C_off, factor patterns, the host
// ILUT factor, level sets and the level programs the device kernels execute.
//
// Paper passages: Sec. 2.2.1 (classification, relabelling, Eq. equ22), Sec. 3.1 (level
// scheduling analysis, L\U stored in the pattern), Sec. 3.2 (local blocks Eq. localA,
// factor extraction L_B, U_B, L_S, U_S, W, Z, the off-diagonal blocks of S, Eq. SS).
#include <algorithm>
#include <chrono>
#include <atomic>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>

#include "handle.h"
#include "stream_layout.h"

static_assert(__BYTE_ORDER__ == __ORDER_LITTLE_ENDIAN__, "streams are written little-endian, as the device reads them");

namespace ilu2l {

namespace {

// ------------------------------------------------------------------------------------
// validation

// ------------------------------------------------------------------------------------
// level computation on a window of a factor pattern (rows r0..r1-1 of one subdomain,
// local numbering, q0 = the subdomain's first Q row).
//   lower: lev(r) = 0 without entries c in [clo, r), else 1 + max lev(c);
//   upper: from the bottom over entries c in (r, chi).
// Returns the number of levels; lev is indexed by local row.

int window_levels(const FPat& F, int32_t q0, int32_t r0, int32_t r1, int32_t clo, int32_t chi,
                  bool upper, std::vector<int32_t>& lev) {
    int nl = 0;
    if (!upper) {
        for (int32_t r = r0; r < r1; r++) {
            int32_t l = 0;
            for (int32_t k = F.rp[q0 + r]; k < F.rp[q0 + r + 1]; k++) {
                const int32_t c = F.ci[k];
                if (c >= clo && c < r) l = std::max(l, lev[c] + 1);
            }
            lev[r] = l;
            nl = std::max(nl, l + 1);
        }
    } else {
        for (int32_t r = r1 - 1; r >= r0; r--) {
            int32_t l = 0;
            for (int32_t k = F.rp[q0 + r]; k < F.rp[q0 + r + 1]; k++) {
                const int32_t c = F.ci[k];
                if (c > r && c < chi) l = std::max(l, lev[c] + 1);
            }
            lev[r] = l;
            nl = std::max(nl, l + 1);
        }
    }
    return nl;
}

void prog_init(ProgHost& P) {
    P.sub_lvl.assign(1, 0);
    P.lvl_ptr.assign(1, 0);
    P.pptr.assign(1, 0);
    P.prow.clear();
    P.pcol.clear();
    P.psrc.clear();
    P.pdsrc.clear();
    P.scan_lvl.clear();
    P.max_level_rows = 0;
    P.max_levels = 0;
}

void prog_close_level(ProgHost& P) {
    const int32_t rows = (int32_t)P.prow.size() - P.lvl_ptr.back();
    P.max_level_rows = std::max(P.max_level_rows, rows);
    P.lvl_ptr.push_back((int32_t)P.prow.size());
}

// Host setups running in this process; each takes its share of the hardware threads, so
// that concurrent setups (several requests being served) do not oversubscribe the cores.
std::atomic<int> g_setups{0};

struct SetupCount {
    SetupCount() { g_setups.fetch_add(1); }
    ~SetupCount() { g_setups.fetch_sub(1); }
};

// fn(t, s0, s1) on up to 16 host threads (fewer while other setups run), thread t taking
// the contiguous subdomains [s0, s1); returns the number of ranges used
template <class Fn>
int for_ranges(int32_t p, Fn fn) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned share = std::max(1u, hw / (unsigned)std::max(1, g_setups.load()));
    unsigned nt = std::max(1u, std::min(16u, share));
    nt = std::max(1u, std::min<unsigned>(nt, (unsigned)std::max(p, 1)));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; t++)
        th.emplace_back(fn, (int)t, (int32_t)((int64_t)p * t / nt), (int32_t)((int64_t)p * (t + 1) / nt));
    for (auto& t : th) t.join();
    return (int)nt;
}

// D = the fragments fr[0..nf) (each from prog_init over consecutive subdomain ranges)
// one after the other, their level, row and entry indices shifted; the arrays are sized
// once and every fragment is copied by its own host thread
void prog_concat(ProgHost& D, const std::vector<const ProgHost*>& fr) {
    const size_t nf = fr.size();
    std::vector<size_t> sb(nf + 1, 0), lv(nf + 1, 0), rw(nf + 1, 0), en(nf + 1, 0);
    for (size_t t = 0; t < nf; t++) {
        sb[t + 1] = sb[t] + fr[t]->sub_lvl.size() - 1;
        lv[t + 1] = lv[t] + fr[t]->lvl_ptr.size() - 1;
        rw[t + 1] = rw[t] + fr[t]->prow.size();
        en[t + 1] = en[t] + fr[t]->pcol.size();
    }
    prog_init(D);
    D.sub_lvl.resize(sb[nf] + 1);
    D.lvl_ptr.resize(lv[nf] + 1);
    D.pptr.resize(rw[nf] + 1);
    D.prow.resize(rw[nf]);
    D.pdsrc.resize(rw[nf]);
    D.pcol.resize(en[nf]);
    D.psrc.resize(en[nf]);
    for_ranges((int32_t)nf, [&](int, int32_t t0, int32_t t1) {
        for (int32_t t = t0; t < t1; t++) {
            const ProgHost& F = *fr[t];
            for (size_t i = 1; i < F.sub_lvl.size(); i++) D.sub_lvl[sb[t] + i] = F.sub_lvl[i] + (int32_t)lv[t];
            for (size_t i = 1; i < F.lvl_ptr.size(); i++) D.lvl_ptr[lv[t] + i] = F.lvl_ptr[i] + (int32_t)rw[t];
            for (size_t i = 1; i < F.pptr.size(); i++) D.pptr[rw[t] + i] = F.pptr[i] + (int32_t)en[t];
            std::copy(F.prow.begin(), F.prow.end(), D.prow.begin() + rw[t]);
            std::copy(F.pdsrc.begin(), F.pdsrc.end(), D.pdsrc.begin() + rw[t]);
            std::copy(F.pcol.begin(), F.pcol.end(), D.pcol.begin() + en[t]);
            std::copy(F.psrc.begin(), F.psrc.end(), D.psrc.begin() + en[t]);
        }
    });
    for (size_t t = 0; t < nf; t++) {
        D.max_level_rows = std::max(D.max_level_rows, fr[t]->max_level_rows);
        D.max_levels = std::max(D.max_levels, fr[t]->max_levels);
        for (int32_t e : fr[t]->scan_lvl) D.scan_lvl.push_back(e + (int32_t)lv[t]);
    }
}

// Input checks (CSR shape, sorted unique columns, stored diagonal, partition range). Rows
// are checked on host threads; any bad row gives ILU_ERR_CSR, as a sequential scan would,
// and the partition is checked only when every row is valid.
ilu_status validate(const ilu_csr* A, const int32_t* part, int32_t p) {
    if (!A || !part || p < 1 || A->n < 0 || A->nnz < 0) return ILU_ERR_ARG;
    if (!A->rowptr || (A->nnz > 0 && (!A->colind || !A->val))) return ILU_ERR_ARG;
    const int32_t n = A->n;
    if (A->rowptr[0] != 0 || A->rowptr[n] != A->nnz) return ILU_ERR_CSR;
    std::atomic<int> bad_row{0}, bad_part{0};
    for_ranges(n, [&](int, int32_t i0, int32_t i1) {
        for (int32_t i = i0; i < i1; i++) {
            const int32_t b = A->rowptr[i], e = A->rowptr[i + 1];
            bool ok = e >= b && e <= A->nnz && b >= 0, diag = false;
            for (int32_t q = b; ok && q < e; q++) {
                const int32_t c = A->colind[q];
                if (c < 0 || c >= n || (q > b && c <= A->colind[q - 1])) ok = false;
                diag |= (c == i);
            }
            if (!ok || !diag) {
                bad_row.store(1, std::memory_order_relaxed);
                return;
            }
            if (part[i] < 0 || part[i] >= p) bad_part.store(1, std::memory_order_relaxed);
        }
    });
    if (bad_row.load()) return ILU_ERR_CSR;
    if (bad_part.load()) return ILU_ERR_ARG;
    return ILU_OK;
}

void prog_push_row(ProgHost& P, const FPat& F, int32_t q0, int32_t r, int32_t clo, int32_t chi,
                   bool upper, int32_t base) {
    P.prow.push_back(r - base);
    for (int32_t k = F.rp[q0 + r]; k < F.rp[q0 + r + 1]; k++) {
        const int32_t c = F.ci[k];
        const bool take = upper ? (c > r && c < chi) : (c >= clo && c < chi && c != r);
        if (take) {
            P.pcol.push_back(c - base);
            P.psrc.push_back((int32_t)(F.base + k));
        }
    }
    P.pptr.push_back((int32_t)P.pcol.size());
    P.pdsrc.push_back(upper ? (int32_t)(F.base + F.dpos[q0 + r]) : -1);
}

// Levels [l0, l1) of program S (rows with their entries) appended to program D as levels
// of its own.
void prog_copy_levels(ProgHost& D, const ProgHost& S, int32_t l0, int32_t l1) {
    for (int32_t l = l0; l < l1; l++) {
        for (int32_t k = S.lvl_ptr[l]; k < S.lvl_ptr[l + 1]; k++) {
            D.prow.push_back(S.prow[k]);
            for (int32_t e = S.pptr[k]; e < S.pptr[k + 1]; e++) {
                D.pcol.push_back(S.pcol[e]);
                D.psrc.push_back(S.psrc[e]);
            }
            D.pptr.push_back((int32_t)D.pcol.size());
            D.pdsrc.push_back(S.pdsrc[k]);
        }
        prog_close_level(D);
    }
}

int32_t row_count(const FPat& F, int32_t q0, int32_t r, int32_t clo, int32_t chi, bool upper) {
    int32_t cnt = 0;
    for (int32_t k = F.rp[q0 + r]; k < F.rp[q0 + r + 1]; k++) {
        const int32_t c = F.ci[k];
        cnt += upper ? (c > r && c < chi) : (c >= clo && c < chi && c != r);
    }
    return cnt;
}

// Levels of a triangular window appended to program P (one subdomain). Unit-lower rows
// with no entry leave x unchanged and are not scheduled; upper rows always are (pivot).
int prog_add_tri(ProgHost& P, const FPat& F, int32_t q0, int32_t r0, int32_t r1, int32_t clo,
                 int32_t chi, bool upper, int32_t base, std::vector<int32_t>& lev) {
    if (r1 <= r0) return 0;
    const int nl = window_levels(F, q0, r0, r1, clo, upper ? chi : r1, upper, lev);
    // bucket rows by level, ascending row inside a level
    std::vector<int32_t> cnt(nl + 1, 0);
    for (int32_t r = r0; r < r1; r++) cnt[lev[r] + 1]++;
    for (int l = 0; l < nl; l++) cnt[l + 1] += cnt[l];
    std::vector<int32_t> order(r1 - r0);
    std::vector<int32_t> fillp(cnt.begin(), cnt.end() - 1);
    for (int32_t r = r0; r < r1; r++) order[fillp[lev[r]]++] = r;
    int added = 0;
    for (int l = 0; l < nl; l++) {
        const size_t before = P.prow.size();
        for (int32_t t = cnt[l]; t < cnt[l + 1]; t++) {
            const int32_t r = order[t];
            if (!upper && row_count(F, q0, r, clo, r, false) == 0) continue;
            prog_push_row(P, F, q0, r, clo, upper ? chi : r, upper, base);
        }
        if (P.prow.size() > before) {
            prog_close_level(P);
            added++;
        }
    }
    return added;
}

// One level holding a block product x[r] -= sum M(r, c) x[c], c in [clo, chi).
int prog_add_single(ProgHost& P, const FPat& F, int32_t q0, int32_t r0, int32_t r1, int32_t clo,
                    int32_t chi, int32_t base) {
    const size_t before = P.prow.size();
    for (int32_t r = r0; r < r1; r++) {
        if (row_count(F, q0, r, clo, chi, false) == 0) continue;
        prog_push_row(P, F, q0, r, clo, chi, false, base);
    }
    if (P.prow.size() > before) {
        prog_close_level(P);
        return 1;
    }
    return 0;
}

// ------------------------------------------------------------------------------------
// host ILUT(tau, p) of a local square matrix given by rows of a Q-order CSR window.
// Dual threshold (the paper uses ILUT without defining it, Sec. 4.2; standard reading):
// t_i = tau ||a_i||_2; eliminate pivots k < i in ascending order with fill; drop l_ik
// (and skip its update) when |l_ik| < t_i; afterwards drop |w_j| < t_i and keep the p
// largest of the L part and of the U part (ties: larger |value|, then smaller column);
// the diagonal is always kept; small pivots perturbed as in the ILU(0) kernel.

struct IlutRow {
    std::vector<int32_t> ci;
    std::vector<double> v;
};

int ilut_local(const int32_t* rp, const int32_t* ci, const double* a, int32_t m, double tau,
               int32_t pkeep, double eps, std::vector<IlutRow>& rows, int* npert) {
    rows.assign(m, IlutRow{});
    std::vector<double> w(m, 0.0);
    std::vector<uint8_t> on(m, 0);
    std::vector<int32_t> diagpos(m, 0);
    std::vector<int32_t> lcand, ulist, lkeep;
    std::vector<std::pair<double, int32_t>> sel;
    for (int32_t i = 0; i < m; i++) {
        double nrm2 = 0.0;
        double amax = 0.0;
        for (int32_t q = rp[i]; q < rp[i + 1]; q++) {
            nrm2 += a[q] * a[q];
            amax = std::max(amax, std::fabs(a[q]));
        }
        const double ti = tau * std::sqrt(nrm2);
        lcand.clear();
        ulist.clear();
        lkeep.clear();
        on[i] = 1;
        w[i] = 0.0;
        for (int32_t q = rp[i]; q < rp[i + 1]; q++) {
            const int32_t c = ci[q];
            w[c] = a[q];
            if (c == i) continue;
            on[c] = 1;
            if (c < i) {
                lcand.push_back(c);
                std::push_heap(lcand.begin(), lcand.end(), std::greater<int32_t>());
            } else {
                ulist.push_back(c);
            }
        }
        while (!lcand.empty()) {
            std::pop_heap(lcand.begin(), lcand.end(), std::greater<int32_t>());
            const int32_t k = lcand.back();
            lcand.pop_back();
            const IlutRow& rk = rows[k];
            const double lik = w[k] / rk.v[diagpos[k]];
            if (std::fabs(lik) < ti) {
                w[k] = 0.0;
                on[k] = 0;
                continue;
            }
            w[k] = lik;
            lkeep.push_back(k);
            for (size_t t = (size_t)diagpos[k] + 1; t < rk.ci.size(); t++) {
                const int32_t j = rk.ci[t];
                if (!on[j]) {
                    on[j] = 1;
                    w[j] = 0.0;
                    if (j < i) {
                        lcand.push_back(j);
                        std::push_heap(lcand.begin(), lcand.end(), std::greater<int32_t>());
                    } else {
                        ulist.push_back(j);
                    }
                }
                w[j] -= lik * rk.v[t];
            }
        }
        auto pick = [&](const std::vector<int32_t>& idx, std::vector<std::pair<int32_t, double>>& out) {
            sel.clear();
            for (int32_t j : idx)
                if (std::fabs(w[j]) >= ti) sel.emplace_back(w[j], j);
            auto better = [](const std::pair<double, int32_t>& x, const std::pair<double, int32_t>& y) {
                const double ax = std::fabs(x.first), ay = std::fabs(y.first);
                if (ax != ay) return ax > ay;
                return x.second < y.second;
            };
            if ((int32_t)sel.size() > pkeep) {
                std::nth_element(sel.begin(), sel.begin() + pkeep, sel.end(), better);
                sel.resize(pkeep);
            }
            out.clear();
            for (auto& e : sel) out.emplace_back(e.second, e.first);
            std::sort(out.begin(), out.end());
        };
        std::vector<std::pair<int32_t, double>> lsel, usel;
        pick(lkeep, lsel);
        pick(ulist, usel);
        double uii = w[i];
        const double thr = eps * amax;
        if (eps > 0.0 && std::fabs(uii) < thr) {
            uii = (uii >= 0.0) ? thr : -thr;
            (*npert)++;
        }
        if (uii == 0.0) return ILU_ERR_ZERO_PIVOT;
        IlutRow& ro = rows[i];
        for (auto& e : lsel) {
            ro.ci.push_back(e.first);
            ro.v.push_back(e.second);
        }
        diagpos[i] = (int32_t)ro.ci.size();
        ro.ci.push_back(i);
        ro.v.push_back(uii);
        for (auto& e : usel) {
            ro.ci.push_back(e.first);
            ro.v.push_back(e.second);
        }
        on[i] = 0;
        w[i] = 0.0;
        for (int32_t j : lkeep) {
            on[j] = 0;
            w[j] = 0.0;
        }
        for (int32_t j : ulist) {
            on[j] = 0;
            w[j] = 0.0;
        }
    }
    return ILU_OK;
}

// ------------------------------------------------------------------------------------
// pieces and waves of a streamed program (stream_layout.h)

struct Piece {
    int32_t k;      // packed row (-1: skip record, a hole in a wave)
    int32_t q0, n;  // entries [q0, q0+n) of the row
    bool last;      // applies the pivot inverse
    uint8_t link;   // scan waves: 0 none, kLinkCol (entry `lead` holds the previous row's
                    // value), kLinkSelf (the own slot does)
    int32_t lead;   // with kLinkCol: the entry written first, in position 0 (else -1)
};
struct Wave {
    size_t p0, p1;  // pieces
    bool sync;      // group barrier after the wave
    bool scan;      // a scan wave: width a multiple of 32, warp u holds pieces [32u, 32u + 32)
};
constexpr uint8_t kLinkCol = 1, kLinkSelf = 2;

// Estimated consumer-group cycles of a wave schedule, used to pick between the level and the
// chain schedule of a section: a plain wave costs about one row's latency (operand loads,
// the product, the store), a scan wave the same plus five shuffle rounds, a barrier about
// the rest of a level. (Measured on GB300: a 48-row level with its barrier takes ~400
// cycles, a chained row ~70.)
constexpr double kCostWave = 70.0, kCostScanWave = 260.0, kCostBarrier = 330.0;
// a chunk of the ring: its copy and its hand-over (used to order the subdomains by cost)
constexpr double kCostChunk = 1500.0;
// the shortest chain worth a scan phase
constexpr int32_t kMinChain = 3;

double schedule_cost(const std::vector<Wave>& waves, size_t w0) {
    double c = 0.0;
    for (size_t w = w0; w < waves.size(); w++)
        c += (waves[w].scan ? kCostScanWave : kCostWave) + (waves[w].sync ? kCostBarrier : 0.0);
    return c;
}

// Chain schedule of packed rows [k0, k1) of one subdomain program (a section that starts
// after a group barrier), appended to pieces / waves; every phase ends with a barrier.
//
// Dependencies between the rows follow the program order: a row reads its columns and its
// own slot (after the last earlier writer of each) and overwrites its own slot (after every
// earlier reader of it since that write). A phase takes the rows whose dependencies are all
// done. From them it grows chains: a row joins the end of a chain when everything it needs
// is done except the chain's last row, whose value it reads through one column or its own
// slot (the link), or earlier rows of the same chain whose slots it only overwrites.
// Such a chain is a first-order linear recurrence, x_i = a_i + b_i x_{i-1}, which a warp
// solves 32 rows at a time by a prefix composition of the affine maps (the scan waves of
// the device). When the longest chain is at least kMinChain rows the phase runs the chains
// (single-piece rows only; longest first, each on the warp with the fewest rows, as far
// as the longest chain's wave count allows); otherwise the ready rows run as one level
// (plain waves, sub-levels for rows split into pieces). Chains of one phase touch
// disjoint state, so the warps need no synchronisation until the phase's barrier.
void phase_schedule(const ProgHost& P, int32_t k0, int32_t k1, int32_t RW, uint32_t nt,
                    std::vector<int32_t>& lw, std::vector<std::vector<int32_t>>& rd,
                    std::vector<Piece>& pieces, std::vector<Wave>& waves) {
    const int32_t m = k1 - k0;
    if (m <= 0) return;
    struct Dep {
        int32_t d;
        int8_t kind;  // 0: d read the slot this row overwrites; kLinkCol: reads d's slot
                      // through entry q; kLinkSelf: reads d's value in its own slot
        int32_t q;
    };
    std::vector<int32_t> dptr((size_t)m + 1, 0);
    std::vector<Dep> deps;
    std::vector<int32_t> touched;
    for (int32_t i = 0; i < m; i++) {
        const int32_t k = k0 + i;
        dptr[i] = (int32_t)deps.size();
        const int32_t a = P.pptr[k], n = P.pptr[k + 1] - a, w = P.prow[k];
        for (int32_t q = 0; q < n; q++) {
            const int32_t c = P.pcol[a + q];
            if (lw[c] >= 0) deps.push_back({lw[c], (int8_t)kLinkCol, q});
        }
        if (lw[w] >= 0) deps.push_back({lw[w], (int8_t)kLinkSelf, -1});
        for (int32_t r : rd[w])
            if (r != i) deps.push_back({r, 0, -1});
        for (int32_t q = 0; q < n; q++) {
            const int32_t c = P.pcol[a + q];
            rd[c].push_back(i);
            touched.push_back(c);
        }
        rd[w].clear();
        lw[w] = i;
        touched.push_back(w);
    }
    dptr[m] = (int32_t)deps.size();
    for (int32_t c : touched) {  // leave the slot maps clean for the next section
        lw[c] = -1;
        rd[c].clear();
    }
    // successors (distinct), open dependency counts, heights (longest path to the end)
    std::vector<int32_t> sptr((size_t)m + 1, 0), succ, left(m, 0), h(m, 1), np(m, 1);
    {
        std::vector<int32_t> seen(m, -1);
        std::vector<std::pair<int32_t, int32_t>> edges;
        for (int32_t i = 0; i < m; i++)
            for (int32_t e = dptr[i]; e < dptr[i + 1]; e++) {
                const int32_t d = deps[e].d;
                if (seen[d] == i) continue;
                seen[d] = i;
                edges.push_back({d, i});
                left[i]++;
            }
        for (auto& ed : edges) sptr[ed.first + 1]++;
        for (int32_t i = 0; i < m; i++) sptr[i + 1] += sptr[i];
        succ.resize(edges.size());
        std::vector<int32_t> fill(sptr.begin(), sptr.end() - 1);
        for (auto& ed : edges) succ[fill[ed.first]++] = ed.second;
    }
    for (int32_t i = m - 1; i >= 0; i--)
        for (int32_t e = sptr[i]; e < sptr[i + 1]; e++) h[i] = std::max(h[i], 1 + h[succ[e]]);
    for (int32_t i = 0; i < m; i++) {
        const int32_t n = P.pptr[k0 + i + 1] - P.pptr[k0 + i];
        np[i] = std::max(1, (n + RW - 1) / RW);
    }
    std::vector<char> done(m, 0), taken(m, 0);
    std::vector<int32_t> chain_of(m, -1), link(m, 0), lead(m, -1), ready, next_ready;
    for (int32_t i = 0; i < m; i++)
        if (left[i] == 0) ready.push_back(i);
    const uint32_t W = std::max(1u, nt / 32);
    int32_t remaining = m;
    std::vector<std::vector<int32_t>> chains;
    auto finish = [&](int32_t i) {
        done[i] = 1;
        remaining--;
        for (int32_t e = sptr[i]; e < sptr[i + 1]; e++)
            if (--left[succ[e]] == 0) next_ready.push_back(succ[e]);
    };
    while (remaining > 0) {
        std::vector<int32_t> R;
        for (int32_t i : ready)
            if (!done[i]) R.push_back(i);
        for (int32_t i : next_ready)
            if (!done[i]) R.push_back(i);
        next_ready.clear();
        std::sort(R.begin(), R.end());
        R.erase(std::unique(R.begin(), R.end()), R.end());
        if (R.empty()) break;  // unreachable: the program order is a topological order
        std::stable_sort(R.begin(), R.end(), [&](int32_t a, int32_t b) { return h[a] > h[b]; });
        // grow chains
        chains.clear();
        size_t lmax = 0;
        for (int32_t i0 : R) {
            if (np[i0] != 1 || taken[i0]) continue;
            const int32_t cid = (int32_t)chains.size();
            chains.push_back({i0});
            taken[i0] = 1;
            chain_of[i0] = cid;
            link[i0] = 0;
            lead[i0] = -1;
            int32_t tail = i0;
            for (;;) {
                int32_t best = -1, bl = 0, bq = -1;
                for (int32_t e = sptr[tail]; e < sptr[tail + 1]; e++) {
                    const int32_t c = succ[e];
                    if (taken[c] || done[c] || np[c] != 1) continue;
                    bool ok = true;
                    int32_t lk = 0, lq = -1;
                    for (int32_t f = dptr[c]; f < dptr[c + 1] && ok; f++) {
                        const Dep& D = deps[f];
                        if (done[D.d]) continue;
                        if (D.d == tail && D.kind == (int8_t)kLinkCol) {
                            lk = kLinkCol;
                            lq = D.q;
                        } else if (D.d == tail && D.kind == (int8_t)kLinkSelf) {
                            lk = kLinkSelf;
                        } else if (!(D.kind == 0 && taken[D.d] && chain_of[D.d] == cid)) {
                            ok = false;
                        }
                    }
                    if (ok && (best < 0 || h[c] > h[best])) {
                        best = c;
                        bl = lk;
                        bq = lq;
                    }
                }
                if (best < 0) break;
                chains[cid].push_back(best);
                taken[best] = 1;
                chain_of[best] = cid;
                link[best] = bl;
                lead[best] = bq;
                tail = best;
            }
            lmax = std::max(lmax, chains[cid].size());
        }
        if ((int32_t)lmax < kMinChain) {
            // a plain level: every ready row, sub-level j holding piece j of each row
            for (auto& ch : chains)
                for (int32_t i : ch) taken[i] = 0, chain_of[i] = -1;
            int32_t npm = 1;
            for (int32_t i : R) npm = std::max(npm, np[i]);
            std::sort(R.begin(), R.end());
            for (int32_t j = 0; j < npm; j++) {
                std::vector<Piece> sub;
                for (int32_t i : R) {
                    const int32_t n = P.pptr[k0 + i + 1] - P.pptr[k0 + i];
                    if (j < np[i]) sub.push_back({k0 + i, j * RW, std::min(RW, n - j * RW), j == np[i] - 1, 0, -1});
                }
                if (!waves.empty()) waves.back().sync = true;
                for (size_t t = 0; t < sub.size(); t += nt) {
                    const size_t t1 = std::min(sub.size(), t + nt);
                    waves.push_back({pieces.size() + t, pieces.size() + t1, false, false});
                }
                pieces.insert(pieces.end(), sub.begin(), sub.end());
            }
            waves.back().sync = true;
            for (int32_t i : R) finish(i);
            ready.clear();
            continue;
        }
        // a scan phase: chains onto warps, longest first, each on the least loaded warp,
        // within the longest chain's wave count; chains that do not fit wait
        std::vector<size_t> order(chains.size());
        for (size_t c = 0; c < order.size(); c++) order[c] = c;
        std::stable_sort(order.begin(), order.end(),
                         [&](size_t a, size_t b) { return chains[a].size() > chains[b].size(); });
        const size_t cap = 32 * ((lmax + 31) / 32);
        std::vector<std::vector<int32_t>> seq(W);
        for (size_t c : order) {
            size_t u = 0;
            for (size_t v = 1; v < W; v++)
                if (seq[v].size() < seq[u].size()) u = v;
            if (seq[u].size() + chains[c].size() <= cap) {
                seq[u].insert(seq[u].end(), chains[c].begin(), chains[c].end());
            } else {
                for (int32_t i : chains[c]) taken[i] = 0, chain_of[i] = -1;
            }
        }
        size_t used = 0, len = 0;
        for (size_t u = 0; u < W; u++)
            if (!seq[u].empty()) used = u + 1, len = std::max(len, seq[u].size());
        const size_t nwv = (len + 31) / 32;
        for (size_t wv = 0; wv < nwv; wv++) {
            const size_t p0 = pieces.size();
            for (size_t u = 0; u < used; u++)
                for (size_t l = 0; l < 32; l++) {
                    const size_t pos = 32 * wv + l;
                    if (pos < seq[u].size()) {
                        const int32_t i = seq[u][pos];
                        const int32_t n = P.pptr[k0 + i + 1] - P.pptr[k0 + i];
                        pieces.push_back({k0 + i, 0, n, true, (uint8_t)link[i], lead[i]});
                    } else {
                        pieces.push_back({-1, 0, 0, false, 0, -1});
                    }
                }
            waves.push_back({p0, pieces.size(), false, true});
        }
        waves.back().sync = true;
        for (size_t u = 0; u < used; u++)
            for (int32_t i : seq[u]) {
                taken[i] = 0;
                chain_of[i] = -1;
                finish(i);
            }
        ready = R;
    }
}

}  // namespace

// ====================================================================================
// chunked streams (stream_layout.h)

bool build_stream(const ProgHost& P, int32_t p, int idx_bytes, int x_bytes, int val_bytes, uint32_t chunk,
                  StreamHost& S, int chain_sched) {
    S.blob.clear();
    S.ch0.assign(1, 0);
    S.voff.clear();
    S.vsrc.clear();
    S.doff.clear();
    S.dsrc.clear();
    S.chunk = chunk;
    S.idx_bytes = idx_bytes;
    S.val_bytes = val_bytes;
    S.x_bytes = x_bytes;
    S.levels = (int64_t)P.lvl_ptr.size() - 1;
    S.rows = (int64_t)P.prow.size();
    S.entries = (int64_t)P.pcol.size();
    // record width: 4 entries unless many rows are longer; longer rows are split into
    // pieces run in consecutive sub-levels (intermediate pieces with a unit pivot)
    int64_t longer = 0;
    for (size_t k = 0; k + 1 < P.pptr.size(); k++) longer += (P.pptr[k + 1] - P.pptr[k]) > 4;
    S.rw = (longer * 20 <= (int64_t)P.prow.size()) ? 4 : 16;
    const int32_t RW = S.rw;
    const RecLayout RL = rec_layout((uint32_t)S.rw, (uint32_t)val_bytes, (uint32_t)x_bytes);
    S.rec_bytes = RL.bytes;
    // a whole wave (one record per consumer thread) must fit one chunk
    const int nt_fit = (int)(((chunk - kChunkHdr - 16) / RL.bytes) / 32 * 32);
    if (nt_fit < 32 || chunk > (1u << 20)) return false;
    S.nt = std::min(S.nt, std::min(nt_fit, kMaxConsumers));
    const uint32_t nt = (uint32_t)S.nt;
    // Barrier elimination. A sub-level joins the current barrier-free stretch (no group
    // barrier before it) when each of its pieces can run on one consumer thread that
    // already holds, within the stretch, everything the piece touches -- the writer of
    // every value it reads (its columns and its own slot), and every earlier reader of
    // the slot it overwrites -- and no two pieces need the same thread. Program order on
    // that thread then replaces the barrier; pieces touching nothing written or read in
    // the stretch go to idle threads. Each piece sits at its thread's position in the
    // wave, skip records filling the holes. Chains -- runs of rows each depending on the
    // previous one, as along a subdomain's interface -- thus run as one thread's sequence
    // instead of one barrier per row. Otherwise the previous wave ends with a barrier and
    // the sub-level starts a new stretch, its pieces spread over the threads in order.
    int32_t maxpos = 0;
    for (int32_t r : P.prow) maxpos = std::max(maxpos, r);
    for (int32_t c : P.pcol) maxpos = std::max(maxpos, c);
    // Subdomains are independent: host threads pack contiguous ranges of them into
    // fragments (offsets relative to the fragment), appended in subdomain order below.
    struct Frag {
        rawvec<uint8_t> blob;
        std::vector<int32_t> nch;  // chunks of each subdomain of the range
        rawvec<int64_t> voff, doff;
        rawvec<int32_t> vsrc, dsrc;
        int64_t waves = 0, segments = 0, records = 0, skips = 0, max_barriers = 0, max_levels_sub = 0;
        int64_t max_scan_waves = 0, max_steps = 0, chain_sections = 0;
        std::vector<double> cost;  // estimated consumer cycles of each subdomain of the range
        bool ok = true;
    };
    std::vector<Frag> frag(16);
    const int nfrag = for_ranges(p, [&](int ti, int32_t s0, int32_t s1) {
        Frag& F = frag[ti];
        auto put = [&](size_t off, uint32_t v, int bytes) {  // little-endian, like the device
            if (bytes == 4)
                std::memcpy(&F.blob[off], &v, 4);
            else
                for (int b = 0; b < bytes; b++) F.blob[off + b] = (uint8_t)(v >> (8 * b));
        };
        // per slot, within the current stretch: writer thread, reader thread (-2: several)
        std::vector<int32_t> wep((size_t)maxpos + 1, -1), wth((size_t)maxpos + 1, -1);
        std::vector<int32_t> rep((size_t)maxpos + 1, -1), rth((size_t)maxpos + 1, -1);
        std::vector<int32_t> used(nt), assign;
        int32_t epoch = 0;
        std::vector<Piece> pieces;
        std::vector<Wave> waves;
        std::vector<Piece> sub;
        auto mark = [&](const Piece& pc, int32_t t) {
            auto rd = [&](int32_t pos) {
                if (rep[pos] != epoch) {
                    rep[pos] = epoch;
                    rth[pos] = t;
                } else if (rth[pos] != t) {
                    rth[pos] = -2;
                }
            };
            for (int32_t q = 0; q < pc.n; q++) rd(P.pcol[P.pptr[pc.k] + pc.q0 + q]);
            const int32_t w = P.prow[pc.k];
            rd(w);
            wep[w] = epoch;
            wth[w] = t;
        };
        // slot maps of the chain schedule (all -1 / empty between sections)
        std::vector<int32_t> ch_lw;
        std::vector<std::vector<int32_t>> ch_rd;
        if (!P.scan_lvl.empty()) {
            ch_lw.assign((size_t)maxpos + 1, -1);
            ch_rd.resize((size_t)maxpos + 1);
        }
        std::vector<Piece> alt_pieces;
        std::vector<Wave> alt_waves;
        // the level schedule of levels [ea, eb) of the current subdomain (barrier elimination
        // above), appended to pieces / waves
        auto level_schedule = [&](int32_t ea, int32_t eb) {
            for (int32_t e = ea; e < eb; e++) {
                const int32_t k0 = P.lvl_ptr[e], k1 = P.lvl_ptr[e + 1];
                int32_t np = 1;
                for (int32_t k = k0; k < k1; k++) np = std::max(np, (P.pptr[k + 1] - P.pptr[k] + RW - 1) / RW);
                for (int32_t j = 0; j < np; j++) {  // sub-level j: piece j of every row that has one
                    sub.clear();
                    for (int32_t k = k0; k < k1; k++) {
                        const int32_t n = P.pptr[k + 1] - P.pptr[k];
                        const int32_t npk = std::max(1, (n + RW - 1) / RW);
                        if (j < npk) sub.push_back({k, j * RW, std::min(RW, n - j * RW), j == npk - 1, 0, -1});
                    }
                    bool merge = !waves.empty() && sub.size() <= nt;
                    if (merge) {
                        std::fill(used.begin(), used.end(), -1);
                        assign.assign(sub.size(), -1);
                        for (size_t i = 0; i < sub.size() && merge; i++) {
                            const Piece& pc = sub[i];
                            int32_t t = -1;
                            auto need = [&](int32_t u) {
                                if (u == -2 || (t >= 0 && t != u)) merge = false;
                                t = u;
                            };
                            for (int32_t q = 0; q < pc.n; q++) {
                                const int32_t c = P.pcol[P.pptr[pc.k] + pc.q0 + q];
                                if (wep[c] == epoch) need(wth[c]);
                            }
                            const int32_t w = P.prow[pc.k];
                            if (wep[w] == epoch) need(wth[w]);
                            if (rep[w] == epoch) need(rth[w]);
                            if (!merge) break;
                            if (t >= 0) {
                                if (used[t] >= 0) {
                                    merge = false;
                                    break;
                                }
                                used[t] = (int32_t)i;
                                assign[i] = t;
                            }
                        }
                        if (merge) {  // free pieces onto the lowest idle threads
                            uint32_t t = 0;
                            for (size_t i = 0; i < sub.size(); i++) {
                                if (assign[i] >= 0) continue;
                                while (used[t] >= 0) t++;
                                used[t] = (int32_t)i;
                                assign[i] = (int32_t)t;
                            }
                        }
                    }
                    if (merge) {
                        uint32_t width = 0;
                        for (int32_t a : assign) width = std::max(width, (uint32_t)a + 1);
                        const size_t p0 = pieces.size();
                        for (uint32_t t = 0; t < width; t++) {
                            if (used[t] >= 0) {
                                const Piece& pc = sub[(size_t)used[t]];
                                pieces.push_back(pc);
                                mark(pc, (int32_t)t);
                            } else {
                                pieces.push_back({-1, 0, 0, false, 0, -1});
                            }
                        }
                        waves.push_back({p0, pieces.size(), false, false});
                    } else {
                        if (!waves.empty()) waves.back().sync = true;
                        epoch++;
                        for (size_t t = 0; t < sub.size(); t += nt) {
                            const size_t t1 = std::min(sub.size(), t + nt);
                            waves.push_back({pieces.size() + t, pieces.size() + t1, false, false});
                        }
                        for (size_t i = 0; i < sub.size(); i++) mark(sub[i], (int32_t)(i % nt));
                        pieces.insert(pieces.end(), sub.begin(), sub.end());
                    }
                }
            }
        };
        for (int32_t s = s0; s < s1; s++) {
            // pieces and waves of this subdomain, in program order
            pieces.clear();
            waves.clear();
            epoch++;
            int64_t nchunks = 0;
            F.max_levels_sub = std::max<int64_t>(F.max_levels_sub, P.sub_lvl[s + 1] - P.sub_lvl[s]);
            const int32_t e_end = P.sub_lvl[s + 1];
            const int32_t e_sec = (P.scan_lvl.empty() || chain_sched == 1)
                                      ? e_end
                                      : std::max(P.sub_lvl[s], std::min(P.scan_lvl[s], e_end));
            level_schedule(P.sub_lvl[s], e_sec);
            if (e_sec < e_end) {
                // the chain section: both schedules after a barrier, the cheaper one kept
                if (!waves.empty()) waves.back().sync = true;
                epoch++;
                const size_t p_mark = pieces.size(), w_mark = waves.size();
                level_schedule(e_sec, e_end);
                if (waves.size() > w_mark) waves.back().sync = true;
                const double c_level = schedule_cost(waves, w_mark);
                alt_pieces.assign(pieces.begin() + (std::ptrdiff_t)p_mark, pieces.end());
                alt_waves.assign(waves.begin() + (std::ptrdiff_t)w_mark, waves.end());
                pieces.resize(p_mark);
                waves.resize(w_mark);
                phase_schedule(P, P.lvl_ptr[e_sec], P.lvl_ptr[e_end], RW, nt, ch_lw, ch_rd, pieces, waves);
                const double c_chain = schedule_cost(waves, w_mark);
                if (chain_sched != 2 && c_level <= c_chain) {
                    pieces.resize(p_mark);
                    waves.resize(w_mark);
                    pieces.insert(pieces.end(), alt_pieces.begin(), alt_pieces.end());
                    waves.insert(waves.end(), alt_waves.begin(), alt_waves.end());
                } else {
                    F.chain_sections++;
                }
            }
            if (!waves.empty()) waves.back().sync = true;
            int64_t barriers = 0, scans = 0;
            for (const Wave& W : waves) barriers += W.sync, scans += W.scan;
            F.max_barriers = std::max(F.max_barriers, barriers);
            F.max_scan_waves = std::max(F.max_scan_waves, scans);
            F.max_steps = std::max(F.max_steps, barriers + scans);
            F.waves += (int64_t)waves.size();
            // Pack the waves into chunks as segments: runs of consecutive waves of one width
            // (a narrower wave joins when the padding at most doubles it), never crossing a
            // barrier or a chunk.
            struct Seg {
                size_t w0, w1;
                uint32_t width;
                bool barrier;
                bool scan;
                bool each;  // a barrier after every wave
            };
            std::vector<Seg> segs;
            size_t wi = 0;
            while (wi < waves.size()) {
                segs.clear();
                size_t recs = 0;
                auto fits = [&](size_t nseg, size_t nrec) {
                    return kChunkHdr + al((uint32_t)(kSegEntry * nseg), 16) + nrec * RL.bytes <= chunk;
                };
                while (wi < waves.size()) {
                    const uint32_t ww = (uint32_t)(waves[wi].p1 - waves[wi].p0);
                    // a plain wave followed by a barrier starts a run of levels (a barrier after
                    // every wave) that later such waves join; other segments end at a barrier
                    const bool level = waves[wi].sync && !waves[wi].scan;
                    const bool open = !segs.empty() && (segs.back().each ? level : !segs.back().barrier);
                    const bool join = open && segs.back().w1 - segs.back().w0 < kSegMaxWaves &&
                                      segs.back().scan == waves[wi].scan &&
                                      (ww == segs.back().width || (ww < segs.back().width && segs.back().width <= 2 * ww));
                    if (join) {
                        if (!fits(segs.size(), recs + segs.back().width)) break;
                        segs.back().w1 = wi + 1;
                        recs += segs.back().width;
                    } else {
                        if (!fits(segs.size() + 1, recs + ww)) break;
                        segs.push_back({wi, wi + 1, ww, false, waves[wi].scan, level});
                        recs += ww;
                    }
                    if (waves[wi].sync && !segs.back().each) segs.back().barrier = true;
                    wi++;
                }
                if (segs.empty()) {  // a wave wider than a chunk (excluded by nt_fit)
                    F.ok = false;
                    return;
                }
                const size_t cb = F.blob.size();
                F.blob.resize(cb + chunk, 0);
                nchunks++;
                F.segments += (int64_t)segs.size();
                put(cb, (uint32_t)segs.size(), 4);
                size_t roff = kChunkHdr + al((uint32_t)(kSegEntry * segs.size()), 16);
                for (size_t g = 0; g < segs.size(); g++) {
                    const Seg& G = segs[g];
                    put(cb + kChunkHdr + kSegEntry * g, (uint32_t)(roff / 16) | (G.width << 16), 4);
                    put(cb + kChunkHdr + kSegEntry * g + 4,
                        (uint32_t)(G.w1 - G.w0) | (G.barrier ? kSegBarrier : 0u) | (G.scan ? kSegScan : 0u) |
                            (G.each ? kSegSyncEach : 0u), 4);
                    for (size_t w = G.w0; w < G.w1; w++) {
                        const Wave& W = waves[w];
                        for (uint32_t t = 0; t < G.width; t++) {
                            const size_t rb = cb + roff;
                            roff += RL.bytes;
                            F.records++;
                            const Piece* pc = (W.p0 + t < W.p1) ? &pieces[W.p0 + t] : nullptr;
                            if (!pc || pc->k < 0) {  // skip record: reads slot 0, stores nothing
                                F.skips++;
                                put(rb, kRecSkip, 4);
                                continue;
                            }
                            const uint32_t row_off = (uint32_t)P.prow[pc->k] * (uint32_t)x_bytes;
                            const uint32_t lbits = pc->link == kLinkCol ? kRecLinkCol : pc->link == kLinkSelf ? kRecLinkSelf : 0u;
                            put(rb, (uint32_t)P.prow[pc->k] | ((uint32_t)pc->n << 24) | lbits, 4);  // row | n | link
                            F.doff.push_back((int64_t)(rb + RL.dinv));
                            F.dsrc.push_back(pc->last ? P.pdsrc[pc->k] : -1);  // -1: the pack writes 1
                            for (int32_t q = 0; q < RW; q++) {
                                if (q >= pc->n) {  // unused entry: the row's own slot times a zero value
                                    put(rb + RL.col + (size_t)q * 4, row_off, 4);
                                    continue;
                                }
                                // with a column link the linked entry comes first, the others
                                // keep their order
                                int32_t qq = q;
                                if (pc->link == kLinkCol && pc->lead >= 0) qq = (q == 0) ? pc->lead : (q <= pc->lead ? q - 1 : q);
                                const int32_t src = P.pptr[pc->k] + pc->q0 + qq;
                                put(rb + RL.col + (size_t)q * 4, (uint32_t)P.pcol[src] * (uint32_t)x_bytes, 4);
                                F.voff.push_back((int64_t)(rb + RL.val + (size_t)q * val_bytes));
                                F.vsrc.push_back(P.psrc[src]);
                            }
                        }
                    }
                }
            }
            F.nch.push_back((int32_t)nchunks);
            F.cost.push_back(schedule_cost(waves, 0) + kCostChunk * (double)nchunks);
        }
    });
    // the fragments one after the other: arrays sized once, one host thread per fragment
    S.waves = S.segments = S.records = S.skips = S.max_barriers = S.max_levels_sub = 0;
    S.max_scan_waves = S.max_steps = S.chain_sections = 0;
    std::vector<size_t> nb(nfrag + 1, 0), nv(nfrag + 1, 0), nd(nfrag + 1, 0);
    for (int t = 0; t < nfrag; t++) {
        const Frag& F = frag[t];
        if (!F.ok) return false;
        nb[t + 1] = nb[t] + F.blob.size();
        nv[t + 1] = nv[t] + F.voff.size();
        nd[t + 1] = nd[t] + F.doff.size();
        for (int32_t c : F.nch) S.ch0.push_back(S.ch0.back() + c);
        S.waves += F.waves;
        S.segments += F.segments;
        S.records += F.records;
        S.skips += F.skips;
        S.max_barriers = std::max(S.max_barriers, F.max_barriers);
        S.max_levels_sub = std::max(S.max_levels_sub, F.max_levels_sub);
        S.max_scan_waves = std::max(S.max_scan_waves, F.max_scan_waves);
        S.max_steps = std::max(S.max_steps, F.max_steps);
        S.chain_sections += F.chain_sections;
    }
    {   // launch order: the most expensive subdomain first (ties: lower index)
        std::vector<double> cost;
        for (int t = 0; t < nfrag; t++) cost.insert(cost.end(), frag[t].cost.begin(), frag[t].cost.end());
        S.order.resize(cost.size());
        for (size_t i = 0; i < cost.size(); i++) S.order[i] = (int32_t)i;
        std::stable_sort(S.order.begin(), S.order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
    }
    S.blob.resize(nb[nfrag]);
    S.voff.resize(nv[nfrag]);
    S.vsrc.resize(nv[nfrag]);
    S.doff.resize(nd[nfrag]);
    S.dsrc.resize(nd[nfrag]);
    for_ranges(nfrag, [&](int, int32_t t0, int32_t t1) {
        for (int32_t t = t0; t < t1; t++) {
            const Frag& F = frag[t];
            const int64_t base = (int64_t)nb[t];
            std::copy(F.blob.begin(), F.blob.end(), S.blob.begin() + nb[t]);
            for (size_t i = 0; i < F.voff.size(); i++) S.voff[nv[t] + i] = F.voff[i] + base;
            std::copy(F.vsrc.begin(), F.vsrc.end(), S.vsrc.begin() + nv[t]);
            for (size_t i = 0; i < F.doff.size(); i++) S.doff[nd[t] + i] = F.doff[i] + base;
            std::copy(F.dsrc.begin(), F.dsrc.end(), S.dsrc.begin() + nd[t]);
        }
    });
    if (S.blob.empty()) S.blob.resize(16, 0);
    return true;
}

// ====================================================================================

// ---- the autotuner's process-wide record ---------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<uint64_t, std::array<int32_t, PR_COUNT>> g_tune;

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(uint64_t v) {
        for (int b = 0; b < 8; b++) {
            h ^= (v >> (8 * b)) & 0xFF;
            h *= 1099511628211ull;
        }
    }
};
}  // namespace

// Options that shape the programs, the problem's sizes, each program's level structure, the
// subdomains' row ranges and the local patterns (row pointers, every 64th column index).
uint64_t tune_key(const Handle& h) {
    Fnv f;
    const ilu_opts& o = h.o;
    for (int64_t v : {(int64_t)h.n, h.nnz, (int64_t)h.p, (int64_t)h.variant, (int64_t)h.form, (int64_t)h.prec,
                      (int64_t)h.kB, (int64_t)h.kS, (int64_t)o.fill_level, (int64_t)o.ordering, (int64_t)o.l1_block,
                      (int64_t)o.chain_sched, (int64_t)o.inner_iters, (int64_t)h.chunk, (int64_t)h.idx_bytes,
                      (int64_t)o.ilut_p})
        f.add((uint64_t)v);
    f.add((uint64_t)(o.ilut_tau * 1e12));
    for (int id = 0; id < PR_COUNT; id++) {
        const ProgHost& P = h.prog[id];
        f.add(P.lvl_ptr.size());
        f.add(P.prow.size());
        f.add(P.pcol.size());
    }
    for (int32_t v : h.qoff) f.add((uint64_t)(uint32_t)v);
    for (int32_t v : h.nint) f.add((uint64_t)(uint32_t)v);
    for (int32_t v : h.q_rp) f.add((uint64_t)(uint32_t)v);
    for (size_t i = 0; i < h.q_ci.size(); i += 64) f.add((uint64_t)(uint32_t)h.q_ci[i]);
    return f.h;
}

bool tune_lookup(uint64_t key, int32_t (&nt)[PR_COUNT]) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    for (int i = 0; i < PR_COUNT; i++) nt[i] = it->second[i];
    return true;
}

void tune_store(uint64_t key, const int32_t (&nt)[PR_COUNT]) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::array<int32_t, PR_COUNT> a;
    for (int i = 0; i < PR_COUNT; i++) a[i] = nt[i];
    g_tune[key] = a;
}

// Level sets of the six factor windows (A or L_A, U_A; L_B, U_B; L_S, U_S) in the global
// interior-first numbering, for introspection (Sec. 3.1); built on the first request.
void host_levels(Handle& h) {
    if (h.lev_ready) return;
    const int32_t n = h.n, p = h.p;
    const bool schur = (h.variant != ILU_VARIANT_BJ);  // two-level structure
    for (int w = 0; w < 6; w++) {
        h.lev[w].assign(n, -1);
        h.nlev[w] = 0;
    }
    std::vector<int32_t> lev(h.max_ns + 1, 0);
    for (int32_t s = 0; s < p; s++) {
        const int32_t q0 = h.qoff[s];
        const int32_t ni = h.nint[s];
        const int32_t ns = h.qoff[s + 1] - q0;
        auto glob = [&](int32_t l) { return l < ni ? h.int_ptr[s] + l : h.n1 + h.if_ptr[s] + (l - ni); };
        const FPat& pa = (!schur) ? h.f1 : h.apat;
        for (int w = 0; w < 6; w++) {
            const FPat& F = (w < 2) ? pa : (w < 4 ? h.f1 : h.f2);
            int32_t r0 = 0, r1 = ns, clo = 0, chi = ns;
            if (w == 2 || w == 3) {
                r1 = ni;
                chi = ni;
            } else if (w == 4 || w == 5) {
                r0 = ni;
                clo = ni;
            }
            const int nl = window_levels(F, q0, r0, r1, clo, chi, (w & 1) != 0, lev);
            h.nlev[w] = std::max(h.nlev[w], (r1 > r0) ? nl : 0);
            for (int32_t r = r0; r < r1; r++) h.lev[w][glob(r)] = lev[r];
        }
    }
    h.lev_ready = true;
}

// Reverse Cuthill-McKee (Sec. 3.1: the local block is put in RCM order before its ILU) of
// the graph that the nodes `grp` (original indices, ascending) induce in A, symmetrised:
// a ~ b when a_ab or a_ba is stored, a != b. Each component is searched breadth first from
// its unplaced node of least (degree, index); a node taken from the front of the sequence
// appends its unplaced neighbours by increasing (degree, index); the finished sequence is
// reversed. `grp` (all in subdomain s) is rewritten in that order. `slot` (size n, all -1)
// maps original indices to positions in `grp` while this runs and is left all -1; only
// entries of subdomain s are touched, so subdomains may run on different threads.
static void rcm_group(const ilu_csr* A, const int32_t* part, int32_t s, std::vector<int32_t>& grp,
                      int32_t* slot) {
    const int32_t m = (int32_t)grp.size();
    if (m <= 1) return;
    for (int32_t k = 0; k < m; k++) slot[grp[k]] = k;
    // the edges of the symmetrised graph as sorted, unique (row << 32 | col) keys
    std::vector<uint64_t> key;
    for (int32_t k = 0; k < m; k++) {
        const int32_t i = grp[k];
        for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
            if (part[A->colind[q]] != s) continue;
            const int32_t t = slot[A->colind[q]];
            if (t >= 0 && t != k) {
                key.push_back(((uint64_t)(uint32_t)k << 32) | (uint32_t)t);
                key.push_back(((uint64_t)(uint32_t)t << 32) | (uint32_t)k);
            }
        }
    }
    std::sort(key.begin(), key.end());
    key.erase(std::unique(key.begin(), key.end()), key.end());
    std::vector<int32_t> off(m + 1, 0), nb(key.size());
    for (size_t e = 0; e < key.size(); e++) {
        off[(key[e] >> 32) + 1]++;
        nb[e] = (int32_t)(key[e] & 0xffffffffu);
    }
    for (int32_t k = 0; k < m; k++) off[k + 1] += off[k];
    // labels follow the ascending original index, so (degree, label) orders like
    // (degree, index)
    auto before = [&](int32_t a, int32_t b) {
        const int32_t da = off[a + 1] - off[a], db = off[b + 1] - off[b];
        return da != db ? da < db : a < b;
    };
    std::vector<int32_t> roots(m);
    for (int32_t k = 0; k < m; k++) roots[k] = k;
    std::sort(roots.begin(), roots.end(), before);
    std::vector<char> placed(m, 0);
    std::vector<int32_t> seq;
    seq.reserve(m);
    std::vector<int32_t> fresh;
    size_t next_root = 0;
    while ((int32_t)seq.size() < m) {
        while (placed[roots[next_root]]) next_root++;
        placed[roots[next_root]] = 1;
        seq.push_back(roots[next_root]);
        for (size_t head = seq.size() - 1; head < seq.size(); head++) {
            const int32_t u = seq[head];
            fresh.clear();
            for (int32_t e = off[u]; e < off[u + 1]; e++)
                if (!placed[nb[e]]) {
                    placed[nb[e]] = 1;
                    fresh.push_back(nb[e]);
                }
            std::sort(fresh.begin(), fresh.end(), before);
            seq.insert(seq.end(), fresh.begin(), fresh.end());
        }
    }
    std::vector<int32_t> out(m);
    for (int32_t k = 0; k < m; k++) out[k] = grp[seq[m - 1 - k]];
    for (int32_t k = 0; k < m; k++) slot[grp[k]] = -1;
    grp.swap(out);
}

// Greedy multicolour order of the group `grp` (original indices of subdomain s, ascending):
// in that order each node takes the smallest colour that none of its earlier neighbours in
// the group (a ~ b when a_ab or a_ba is stored, a != b) has; the group is then listed colour
// by colour, ascending index inside a colour (Sec. 3.1: a lower factor in the pattern of A
// gets one level per colour). `slot` as for rcm_group.
static void color_group(const ilu_csr* A, const int32_t* part, int32_t s, std::vector<int32_t>& grp,
                        int32_t* slot) {
    const int32_t m = (int32_t)grp.size();
    if (m <= 1) return;
    for (int32_t k = 0; k < m; k++) slot[grp[k]] = k;
    // neighbour lists of the symmetrised graph, both directions of every stored entry
    std::vector<int32_t> deg(m + 1, 0);
    for (int32_t k = 0; k < m; k++) {
        const int32_t i = grp[k];
        for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
            if (part[A->colind[q]] != s) continue;
            const int32_t t = slot[A->colind[q]];
            if (t >= 0 && t != k) {
                deg[k + 1]++;
                deg[t + 1]++;
            }
        }
    }
    for (int32_t k = 0; k < m; k++) deg[k + 1] += deg[k];
    std::vector<int32_t> nb(deg[m]), fill(deg.begin(), deg.end() - 1);
    for (int32_t k = 0; k < m; k++) {
        const int32_t i = grp[k];
        for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
            if (part[A->colind[q]] != s) continue;
            const int32_t t = slot[A->colind[q]];
            if (t >= 0 && t != k) {
                nb[fill[k]++] = t;
                nb[fill[t]++] = k;
            }
        }
    }
    std::vector<int32_t> colour(m, 0), seen(m + 1, -1);
    int32_t ncol = 0;
    for (int32_t k = 0; k < m; k++) {  // labels ascend with the original index
        for (int32_t e = deg[k]; e < deg[k + 1]; e++)
            if (nb[e] < k) seen[colour[nb[e]]] = k;
        int32_t c = 0;
        while (seen[c] == k) c++;
        colour[k] = c;
        ncol = std::max(ncol, c + 1);
    }
    std::vector<int32_t> start(ncol + 1, 0), out(m);
    for (int32_t k = 0; k < m; k++) start[colour[k] + 1]++;
    for (int32_t c = 0; c < ncol; c++) start[c + 1] += start[c];
    for (int32_t k = 0; k < m; k++) out[start[colour[k]]++] = grp[k];
    for (int32_t k = 0; k < m; k++) slot[grp[k]] = -1;
    grp.swap(out);
}

// Level-k fill pattern of ILU(k) of one local block: rows [q0, q0 + ns) of the Q-order CSR
// (rp, ci; local column indices, sorted, diagonal stored). Stored entries have level 0;
// row r is eliminated with its pivots m < r in ascending order, fill included, and every
// entry u_mj (j > m) already kept in row m gives (r, j) the level lev(r, m) + lev(m, j) + 1;
// the least level wins and levels <= k are kept. While a row is eliminated its columns sit
// in a sorted singly linked list (head = ns), so fill is inserted in place. Output: local
// CSR (orp, oci) and, for the values, the position of each kept entry in the input (-1 =
// fill).
static void iluk_block(const std::vector<int32_t>& rp, const rawvec<int32_t>& ci, int32_t q0, int32_t ns,
                       int k, std::vector<int32_t>& orp, std::vector<int32_t>& oci, std::vector<int64_t>& osrc) {
    const int32_t head = ns;
    std::vector<int32_t> nxt(ns + 1, -1), lev(ns, -1), diag(ns, -1);
    std::vector<int32_t> olev;
    orp.assign(ns + 1, 0);
    oci.clear();
    osrc.clear();
    for (int32_t r = 0; r < ns; r++) {
        // stored entries, already ascending
        int32_t tail = head;
        for (int32_t q = rp[q0 + r]; q < rp[q0 + r + 1]; q++) {
            const int32_t j = ci[q];
            lev[j] = 0;
            nxt[tail] = j;
            tail = j;
        }
        nxt[tail] = ns;  // end marker: ns is never a column
        for (int32_t m = nxt[head]; m < r; m = nxt[m]) {
            const int32_t lm = lev[m];
            int32_t at = m;  // insertion walk starts at the pivot: fill columns are > m
            for (int32_t t = diag[m] + 1; t < orp[m + 1]; t++) {
                const int32_t j = oci[t], l = lm + olev[t] + 1;
                if (l > k) continue;
                if (lev[j] >= 0) {
                    lev[j] = std::min(lev[j], l);
                    continue;
                }
                while (nxt[at] < j) at = nxt[at];
                nxt[j] = nxt[at];
                nxt[at] = j;
                lev[j] = l;
            }
        }
        int32_t q = rp[q0 + r];
        for (int32_t j = nxt[head]; j < ns; j = nxt[j]) {
            if (j == r) diag[r] = (int32_t)oci.size();
            while (q < rp[q0 + r + 1] && ci[q] < j) q++;
            osrc.push_back((q < rp[q0 + r + 1] && ci[q] == j) ? (int64_t)q : -1);
            oci.push_back(j);
            olev.push_back(lev[j]);
            lev[j] = -1;
        }
        orp[r + 1] = (int32_t)oci.size();
    }
}

ilu_status host_setup(Handle& h, const ilu_csr* A, const int32_t* part, int32_t p) {
    SetupCount running;
    ilu_status st = validate(A, part, p);
    if (st != ILU_OK) return st;
    const int32_t n = A->n;
    h.n = n;
    h.p = p;
    h.nnz = A->nnz;
    h.part.assign(part, part + n);

    // ---- classification (Sec. 2.2.1): interface iff coupled to another subdomain in A
    //      or A^T (symmetrised pattern keeps B, E, F block diagonal for any pattern).
    //      Block Jacobi factors each whole A_i (Sec. 2.1): it has no interface.
    h.iface.assign(n, 0);
    if (h.variant != ILU_VARIANT_BJ) {
        int32_t* iface = h.iface.data();
        for_ranges(n, [&](int, int32_t i0, int32_t i1) {  // marks may cross ranges: atomic stores
            for (int32_t i = i0; i < i1; i++)
                for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
                    const int32_t j = A->colind[q];
                    if (part[j] != part[i]) {
                        __atomic_store_n(&iface[i], 1, __ATOMIC_RELAXED);
                        __atomic_store_n(&iface[j], 1, __ATOMIC_RELAXED);
                    }
                }
        });
    }

    // ---- interior-first relabelling (Eq. equ22)
    h.int_ptr.assign(p + 1, 0);
    h.if_ptr.assign(p + 1, 0);
    for (int32_t i = 0; i < n; i++) (h.iface[i] ? h.if_ptr : h.int_ptr)[part[i] + 1]++;
    for (int32_t s = 0; s < p; s++) {
        h.int_ptr[s + 1] += h.int_ptr[s];
        h.if_ptr[s + 1] += h.if_ptr[s];
    }
    h.n1 = h.int_ptr[p];
    h.n2 = n - h.n1;
    h.perm.assign(n, 0);
    h.iperm.assign(n, 0);
    {
        std::vector<int32_t> ci(h.int_ptr.begin(), h.int_ptr.end() - 1);
        std::vector<int32_t> cf(h.if_ptr.begin(), h.if_ptr.end() - 1);
        for (int32_t i = 0; i < n; i++) {
            const int32_t s = part[i];
            const int32_t g = h.iface[i] ? h.n1 + cf[s]++ : ci[s]++;
            h.perm[g] = i;
            h.iperm[i] = g;
        }
    }

    // ---- RCM or colour order inside each group (Sec. 3.1; Algorithm "Block Jacobi ILU on
    //      GPU"): block Jacobi orders all of A_s, the two-level variants its interior nodes
    //      and its interface nodes separately, so A_s keeps its [B F; E C] form
    if (h.o.ordering == ILU_ORDER_RCM || h.o.ordering == ILU_ORDER_COLOR) {
        std::vector<int32_t> slot(n, -1);
        const bool rcm = h.o.ordering == ILU_ORDER_RCM;
        auto work = [&](int32_t s0, int32_t s1) {
            std::vector<int32_t> grp;
            for (int32_t s = s0; s < s1; s++)
                for (int side = 0; side < 2; side++) {
                    const int32_t g0 = side ? h.n1 + h.if_ptr[s] : h.int_ptr[s];
                    const int32_t g1 = side ? h.n1 + h.if_ptr[s + 1] : h.int_ptr[s + 1];
                    grp.assign(h.perm.begin() + g0, h.perm.begin() + g1);
                    if (rcm)
                        rcm_group(A, part, s, grp, slot.data());
                    else
                        color_group(A, part, s, grp, slot.data());
                    for (int32_t k = 0; k < g1 - g0; k++) {
                        h.perm[g0 + k] = grp[k];
                        h.iperm[grp[k]] = g0 + k;
                    }
                }
        };
        for_ranges(p, [&](int, int32_t s0, int32_t s1) { work(s0, s1); });
    }

    // ---- Q order: subdomain s owns [qoff[s], qoff[s+1]) = [interior_s ; interface_s]
    h.qoff.assign(p + 1, 0);
    h.nint.assign(p, 0);
    h.max_ns = 0;
    for (int32_t s = 0; s < p; s++) {
        h.nint[s] = h.int_ptr[s + 1] - h.int_ptr[s];
        const int32_t ns = h.nint[s] + (h.if_ptr[s + 1] - h.if_ptr[s]);
        h.qoff[s + 1] = h.qoff[s] + ns;
        h.max_ns = std::max(h.max_ns, ns);
    }
    h.q_orig.assign(n, 0);
    std::vector<int32_t> loc(n);  // local index of every original node in its subdomain
    for (int32_t s = 0; s < p; s++) {
        const int32_t ni = h.nint[s];
        for (int32_t l = 0; l < ni; l++) {
            const int32_t i = h.perm[h.int_ptr[s] + l];
            h.q_orig[h.qoff[s] + l] = i;
            loc[i] = l;
        }
        for (int32_t l = 0; l < h.if_ptr[s + 1] - h.if_ptr[s]; l++) {
            const int32_t i = h.perm[h.n1 + h.if_ptr[s] + l];
            h.q_orig[h.qoff[s] + ni + l] = i;
            loc[i] = ni + l;
        }
    }

    // ---- local blocks A_s (Eq. localA) in Q order, and C_off (off-diagonal blocks of S,
    //      which equal those of C, Sec. 2.2.2) in interface numbering
    h.q_rp.assign(n + 1, 0);
    h.coff_rp.assign(h.n2 + 1, 0);
    for (int32_t q = 0; q < n; q++) {
        const int32_t i = h.q_orig[q];
        int32_t c_in = 0, c_out = 0;
        for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++)
            (part[A->colind[k]] == part[i] ? c_in : c_out)++;
        h.q_rp[q + 1] = h.q_rp[q] + c_in;
        if (h.iface[i]) h.coff_rp[h.iperm[i] - h.n1 + 1] = c_out;
    }
    for (int32_t r = 0; r < h.n2; r++) h.coff_rp[r + 1] += h.coff_rp[r];
    int64_t nnzQ = h.q_rp[n];
    h.q_ci.resize(nnzQ);
    h.q_v.resize(nnzQ);
    h.q_dpos.assign(n, -1);
    h.coff_ci.resize(h.coff_rp[h.n2]);
    h.coff_v.resize(h.coff_rp[h.n2]);
    h.nnz_coff = h.coff_rp[h.n2];
    // rows are independent from here: host threads fill contiguous row ranges
    for_ranges(n, [&](int, int32_t qa, int32_t qb) {
        std::vector<std::pair<int32_t, double>> row;
        for (int32_t q = qa; q < qb; q++) {
            const int32_t i = h.q_orig[q];
            row.clear();
            double l1 = 0.0;  // l1-BJ (Sec. 4.3): |a_ij| over the other subdomains' columns
            for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) {
                const int32_t j = A->colind[k];
                if (part[j] == part[i])
                    row.emplace_back(loc[j], A->val[k]);
                else
                    l1 += std::fabs(A->val[k]);
            }
            std::sort(row.begin(), row.end(),
                      [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                          return a.first < b.first;
                      });
            int32_t at = h.q_rp[q];
            int32_t s = part[i];
            int32_t lrow = q - h.qoff[s];
            for (auto& e : row) {
                if (e.first == lrow) h.q_dpos[q] = at;
                h.q_ci[at] = e.first;
                h.q_v[at++] = e.second;
            }
            if (h.o.l1_block) h.q_v[h.q_dpos[q]] += l1;
            if (h.iface[i]) {
                row.clear();
                for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) {
                    const int32_t j = A->colind[k];
                    if (part[j] != part[i]) row.emplace_back(h.iperm[j] - h.n1, A->val[k]);
                }
                std::sort(row.begin(), row.end(),
                          [](const std::pair<int32_t, double>& a,
                             const std::pair<int32_t, double>& b) { return a.first < b.first; });
                int32_t at2 = h.coff_rp[h.iperm[i] - h.n1];
                for (auto& e : row) {
                    h.coff_ci[at2] = e.first;
                    h.coff_v[at2++] = e.second;
                }
            }
        }
    });

    // ---- ILU(k) / MILU(k): every local block is stored in its level-k fill pattern with
    //      zeros at the fill positions, so the device ILU(0) / MILU(0) of the stored block
    //      is ILU(k) / MILU(k) of A_s
    if (h.o.fill_level > 0) {
        std::vector<std::vector<int32_t>> brp(p), bci(p);
        std::vector<std::vector<int64_t>> bsrc(p);
        auto work = [&](int32_t s0, int32_t s1) {
            for (int32_t s = s0; s < s1; s++)
                iluk_block(h.q_rp, h.q_ci, h.qoff[s], h.qoff[s + 1] - h.qoff[s], h.o.fill_level, brp[s], bci[s],
                           bsrc[s]);
        };
        for_ranges(p, [&](int, int32_t s0, int32_t s1) { work(s0, s1); });
        int64_t tot = 0;
        for (int32_t s = 0; s < p; s++) tot += (int64_t)bci[s].size();
        if (tot >= (int64_t)INT32_MAX) return ILU_ERR_TOO_LARGE;
        std::vector<int32_t> rp2(n + 1, 0);
        rawvec<int32_t> ci2;
        rawvec<double> v2;
        ci2.reserve(tot);
        v2.reserve(tot);
        for (int32_t s = 0; s < p; s++) {
            const int32_t q0 = h.qoff[s], ns = h.qoff[s + 1] - q0;
            for (int32_t r = 0; r < ns; r++) {
                for (int32_t t = brp[s][r]; t < brp[s][r + 1]; t++) {
                    if (bci[s][t] == r) h.q_dpos[q0 + r] = (int32_t)ci2.size();
                    ci2.push_back(bci[s][t]);
                    v2.push_back(bsrc[s][t] >= 0 ? h.q_v[bsrc[s][t]] : 0.0);
                }
                rp2[q0 + r + 1] = (int32_t)ci2.size();
            }
        }
        h.q_rp.swap(rp2);
        h.q_ci.swap(ci2);
        h.q_v.swap(v2);
        nnzQ = h.q_rp[n];
    }

    // ---- factor patterns and value regions [F1 | F2 | A_local]
    FPat apat;  // views of the local blocks' arrays, final from here on
    apat.rp = h.q_rp.data();
    apat.ci = h.q_ci.data();
    apat.dpos = h.q_dpos.data();
    apat.nnz = nnzQ;
    const bool schur = (h.variant != ILU_VARIANT_BJ);  // two-level structure (SCHUR, RAP)
    const bool rap = (h.variant == ILU_VARIANT_RAP);
    const bool f1_ilut = (h.kB == ILU_FACT_ILUT);
    h.f1_device = !f1_ilut;
    if (!f1_ilut) {
        h.f1 = apat;
        h.f1.base = 0;
    } else {
        // ILUT of B_s (two-level) or of A_s (block Jacobi): on the device (kernels_ilut.cu)
        // unless the handle is analysis-only or asks for the host; the host factorisation
        // below when the device one cannot take the rows (p > 32, a row wider than its table)
        const auto t_ilut = std::chrono::steady_clock::now();
        ilu_status ds = ILU_ERR_UNSUPPORTED;
        if (!h.o.analysis_only && h.o.ilut_setup == 0) ds = device_ilut(h);
        if (ds != ILU_OK && ds != ILU_ERR_UNSUPPORTED) return ds;
        h.ilut_device = (ds == ILU_OK);
        if (!h.ilut_device) {
            std::vector<std::vector<IlutRow>> res(p);
            std::vector<int> stat(p, ILU_OK), pert(p, 0);
            const double tau = h.o.ilut_tau;
            const int32_t pk = h.o.ilut_p;
            const double eps = h.o.pivot_eps;
            auto work = [&](int32_t s0, int32_t s1) {
                std::vector<int32_t> brp, bci;
                std::vector<double> bv;
                for (int32_t s = s0; s < s1; s++) {
                    const int32_t q0 = h.qoff[s];
                    const int32_t m = schur ? h.nint[s] : (h.qoff[s + 1] - q0);
                    brp.assign(m + 1, 0);
                    bci.clear();
                    bv.clear();
                    for (int32_t r = 0; r < m; r++) {
                        for (int32_t k = h.q_rp[q0 + r]; k < h.q_rp[q0 + r + 1]; k++)
                            if (h.q_ci[k] < m) {
                                bci.push_back(h.q_ci[k]);
                                bv.push_back(h.q_v[k]);
                            }
                        brp[r + 1] = (int32_t)bci.size();
                    }
                    stat[s] = ilut_local(brp.data(), bci.data(), bv.data(), m, tau, pk, eps, res[s],
                                         &pert[s]);
                }
            };
            for_ranges(p, [&](int, int32_t s0, int32_t s1) { work(s0, s1); });
            for (int32_t s = 0; s < p; s++) {
                if (stat[s] != ILU_OK) return (ilu_status)stat[s];
                h.npert += pert[s];
            }
            h.f1_rp.assign(n + 1, 0);
            h.f1_dpos.assign(n, -1);
            h.f1_ci.clear();
            h.f1_host_vals.clear();
            for (int32_t s = 0; s < p; s++) {
                const int32_t q0 = h.qoff[s];
                const int32_t ns = h.qoff[s + 1] - q0;
                for (int32_t r = 0; r < ns; r++) {
                    const int32_t q = q0 + r;
                    if (r < (int32_t)res[s].size()) {
                        const IlutRow& ro = res[s][r];
                        for (size_t t = 0; t < ro.ci.size(); t++) {
                            if (ro.ci[t] == r) h.f1_dpos[q] = (int32_t)h.f1_ci.size();
                            h.f1_ci.push_back(ro.ci[t]);
                            h.f1_host_vals.push_back(ro.v[t]);
                        }
                    }
                    h.f1_rp[q + 1] = (int32_t)h.f1_ci.size();
                }
            }
        }
        h.ilut_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_ilut).count();
        h.f1.rp = h.f1_rp.data();
        h.f1.ci = h.f1_ci.data();
        h.f1.dpos = h.f1_dpos.data();
        h.f1.nnz = (int64_t)h.f1_ci.size();
        h.f1.base = 0;
    }
    const int64_t nnz1 = h.f1.nnz;
    h.f2_alias = !(schur && (f1_ilut || h.kS != h.kB));
    if (h.f2_alias) {
        h.f2 = h.f1;
        h.a_base = nnz1;
    } else {
        h.f2 = apat;
        h.f2.base = nnz1;
        h.a_base = nnz1 + nnzQ;
    }
    apat.base = h.a_base;
    h.nvals = h.a_base + nnzQ;
    if (h.nvals >= (int64_t)INT32_MAX) return ILU_ERR_TOO_LARGE;

    // ---- level programs (the introspection level sets are built on demand)
    h.apat = apat;
    h.lev_ready = false;
    for (int pr = 0; pr < PR_COUNT; pr++) prog_init(h.prog[pr]);
    prog_init(h.numprog);
    const bool wz = (h.form == ILU_FORM_WZ);
    // each thread builds the programs of a contiguous range of subdomains; the fragments
    // are appended in subdomain order, so the result equals a sequential build
    std::vector<std::array<ProgHost, PR_COUNT + 1>> frag(16);
    const int nfrag = for_ranges(p, [&](int t, int32_t s0, int32_t s1) {
        std::array<ProgHost, PR_COUNT + 1>& G = frag[t];
        for (auto& P : G) prog_init(P);
        std::vector<int32_t> lev(h.max_ns + 1, 0);
        for (int32_t s = s0; s < s1; s++) {
            const int32_t q0 = h.qoff[s];
            const int32_t ni = h.nint[s];
            const int32_t ns = h.qoff[s + 1] - q0;
            // numeric factorisation schedule: L levels of the pattern of A_s (all local rows)
            {
                ProgHost& N = G[PR_COUNT];
                const int nl = window_levels(apat, q0, 0, ns, 0, ns, false, lev);
                std::vector<std::vector<int32_t>> byl(nl);
                for (int32_t r = 0; r < ns; r++) byl[lev[r]].push_back(r);
                for (int l = 0; l < nl; l++) {
                    for (int32_t r : byl[l]) N.prow.push_back(r);
                    prog_close_level(N);
                }
                N.sub_lvl.push_back((int32_t)N.lvl_ptr.size() - 1);
                N.max_levels = std::max(N.max_levels, nl);
            }
            if (!schur || rap) {  // block Jacobi, or the smoother of the multiplicative variant
                ProgHost& P = G[PR_BJ];
                int a = prog_add_tri(P, h.f1, q0, 0, ns, 0, ns, false, 0, lev);
                a += prog_add_tri(P, h.f1, q0, 0, ns, 0, ns, true, 0, lev);
                P.sub_lvl.push_back((int32_t)P.lvl_ptr.size() - 1);
                P.max_levels = std::max(P.max_levels, a);
            }
            if (schur) {
                // the B parts (L_B, U_B, W, Z): factor_B's factorisation for SCHUR; for RAP the
                // factorisation that defines R and P (Eq. wzinmilu), factor_S's
                const FPat& fb = rap ? h.f2 : h.f1;
                {   // forward and the first local Schur solve in one program (base 0); the
                    // chain section starts at the interface rows (the W or E product)
                    ProgHost& P = G[PR_FWDS];
                    const int32_t l0 = (int32_t)P.lvl_ptr.size() - 1;
                    int a = prog_add_tri(P, fb, q0, 0, ni, 0, ni, false, 0, lev);
                    if (!wz) a += prog_add_tri(P, fb, q0, 0, ni, 0, ni, true, 0, lev);
                    P.scan_lvl.push_back((int32_t)P.lvl_ptr.size() - 1);
                    if (wz)
                        a += prog_add_single(P, fb, q0, ni, ns, 0, ni, 0);
                    else
                        a += prog_add_single(P, apat, q0, ni, ns, 0, ni, 0);
                    const int32_t l1 = (int32_t)P.lvl_ptr.size() - 1;
                    a += prog_add_tri(P, h.f2, q0, ni, ns, ni, ns, false, 0, lev);
                    a += prog_add_tri(P, h.f2, q0, ni, ns, ni, ns, true, 0, lev);
                    P.sub_lvl.push_back((int32_t)P.lvl_ptr.size() - 1);
                    P.max_levels = std::max(P.max_levels, a);
                    // forward alone: f' = L_B^{-1} f then g' = g - W f' (W/Z), or
                    // t = U_B^{-1} L_B^{-1} f then g' = g - E t (E/F) -- the levels before
                    // the local Schur solve above, copied rather than built again
                    ProgHost& F = G[PR_FWD];
                    prog_copy_levels(F, P, l0, l1);
                    F.sub_lvl.push_back((int32_t)F.lvl_ptr.size() - 1);
                    F.max_levels = std::max(F.max_levels, l1 - l0);
                }
                {   // local Schur solve U_S^{-1} L_S^{-1} on the interface part (base ni), one
                    // chain section
                    ProgHost& P = G[PR_S];
                    P.scan_lvl.push_back((int32_t)P.lvl_ptr.size() - 1);
                    int a = prog_add_tri(P, h.f2, q0, ni, ns, ni, ns, false, ni, lev);
                    a += prog_add_tri(P, h.f2, q0, ni, ns, ni, ns, true, ni, lev);
                    P.sub_lvl.push_back((int32_t)P.lvl_ptr.size() - 1);
                    P.max_levels = std::max(P.max_levels, a);
                }
                {   // backward: u = U_B^{-1}(f' - Z y)  (W/Z);  u = U_B^{-1} L_B^{-1}(f - F y) (E/F)
                    ProgHost& P = G[PR_BWD];
                    int a = 0;
                    if (wz) {
                        a += prog_add_single(P, fb, q0, 0, ni, ni, ns, 0);
                    } else {
                        a += prog_add_single(P, apat, q0, 0, ni, ni, ns, 0);
                        a += prog_add_tri(P, fb, q0, 0, ni, 0, ni, false, 0, lev);
                    }
                    a += prog_add_tri(P, fb, q0, 0, ni, 0, ni, true, 0, lev);
                    P.sub_lvl.push_back((int32_t)P.lvl_ptr.size() - 1);
                    P.max_levels = std::max(P.max_levels, a);
                }
            }
        }
    });
    for (int pr = 0; pr <= PR_COUNT; pr++) {
        std::vector<const ProgHost*> fr;
        for (int t = 0; t < nfrag; t++) fr.push_back(&frag[t][pr]);
        prog_concat((pr == PR_COUNT) ? h.numprog : h.prog[pr], fr);
    }

    // ---- chunked streams of the programs the apply runs (TMA fast path)
    if (h.stream_path) {
        h.idx_bytes = 4;
        // working vector (and dinv) in the arithmetic type; values in it or in bfloat16
        const int vb = (h.prec == ILU_PREC_FP64) ? 8 : 4;
        const int valb = (h.prec == ILU_PREC_BF16_STORE) ? 2 : vb;
        if ((int64_t)h.max_ns + 1 >= (1 << 24)) h.stream_path = false;  // the head's row index: 24 bits
        std::vector<int> ids = rap     ? std::vector<int>{PR_BJ, PR_FWDS, PR_BWD}
                               : schur ? std::vector<int>{PR_FWDS, PR_S, PR_BWD}
                                       : std::vector<int>{PR_BJ};
        // consumer group: enough warps for nine levels in ten to run as a single wave
        // (a wave costs about one row's latency whatever its width), at most 128 threads
        for (int id : ids) {
            const ProgHost& P = h.prog[id];
            std::vector<int32_t> wid;
            for (size_t e = 0; e + 1 < P.lvl_ptr.size(); e++) wid.push_back(P.lvl_ptr[e + 1] - P.lvl_ptr[e]);
            int32_t w90 = 1;
            if (!wid.empty()) {
                std::nth_element(wid.begin(), wid.begin() + (wid.size() * 9) / 10, wid.end());
                w90 = wid[(wid.size() * 9) / 10];
            }
            int nt = std::min(128, std::max(32, (w90 + 31) / 32 * 32));
            // programs with a chain section: at least two warps, so that independent chains
            // (the sides of a subdomain's interface) run side by side
            if (!P.scan_lvl.empty()) nt = std::max(nt, 64);
            if (h.o.block_threads) nt = std::max(32, (int)h.o.block_threads);
            h.sh[id].nt = std::min(nt, kMaxConsumers);
        }
        // Ring: two stages of the largest chunk that leaves every subdomain's working
        // vector in shared memory. A chunk boundary costs about 500 cycles and the copy of
        // the next chunk always finishes while the current one runs (measured on the
        // 1024^2 workload: 2 x 32 KB and 4 x 32 KB take the same time, 2 x 64 KB is 4 %
        // faster per apply), so fewer, larger chunks are faster. When the vector cannot stay
        // in shared memory anyway, the largest chunk: the kernels then request only the
        // ring and the rest of the on-chip memory serves the vector as L1.
        const int64_t room = (int64_t)h.smem_optin - 20 * 1024 - 128;
        const int64_t xbytes = (int64_t)(h.max_ns + 1) * vb;
        h.nst = 2;
        h.chunk = 65536;
        for (uint32_t c : {65536u, 32768u, 16384u})
            if (h.nst * (int64_t)c + xbytes <= room) {
                h.chunk = c;
                break;
            }
        // a consumer-group size the autotuner measured for this structure earlier in the process
        h.tune_state = 0;
        if (h.o.autotune && !h.o.block_threads) {
            h.tune_key_v = tune_key(h);
            int32_t nt[PR_COUNT];
            if (tune_lookup(h.tune_key_v, nt)) {
                for (int id : ids)
                    if (nt[id] > 0) h.sh[id].nt = nt[id];
                h.tune_state = 2;
            }
        }
        bool ok = true;
        for (int id : ids) ok = ok && build_stream(h.prog[id], p, h.idx_bytes, vb, valb, h.chunk, h.sh[id], h.o.chain_sched);
        if (!ok) h.stream_path = false;
    }
    return ILU_OK;
}

}  // namespace ilu2l