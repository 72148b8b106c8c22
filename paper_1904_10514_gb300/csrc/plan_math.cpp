// Host-side FP64 construction of the HP2SPH plan tables (see plan_math.h).
#include "plan_math.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#ifndef HPX_ES_WIDTH_FP64
#define HPX_ES_WIDTH_FP64 16
#endif
#ifndef HPX_ES_WIDTH_FP32
#define HPX_ES_WIDTH_FP32 10
#endif

namespace hpx {

namespace {

using cd = std::complex<double>;
const double kPi = 3.14159265358979323846264338327950288;

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

// In-place iterative radix-2 FFT, forward sign e^{-2 pi i jk/n}.
void fft_host(std::vector<cd>& a) {
    const int n = (int)a.size();
    const int lg = ilog2(n);
    for (int i = 0; i < n; ++i) {
        int r = 0;
        for (int b = 0; b < lg; ++b) r |= ((i >> b) & 1) << (lg - 1 - b);
        if (i < r) std::swap(a[i], a[r]);
    }
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len / 2;
        for (int k = 0; k < half; ++k) {
            const double ang = -2.0 * kPi * (double)k / (double)len;
            const cd w(std::cos(ang), std::sin(ang));
            for (int s = 0; s < n; s += len) {
                cd u = a[s + k], v = a[s + k + half] * w;
                a[s + k] = u + v;
                a[s + k + half] = u - v;
            }
        }
    }
}

// theta of north ring j (1-based, j <= 2 N_side), Eq. (healpts).
double ring_theta(int j, int ns) {
    if (j < ns) return 2.0 * std::asin((double)j / (std::sqrt(6.0) * ns));
    return std::acos(2.0 * (2.0 * ns - j) / (3.0 * ns));
}

// Cholesky factorisation (lower) in place, row-major n x n.  Returns false if
// the matrix is not positive definite.
bool cholesky(std::vector<double>& A, int n) {
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        A[(size_t)j * n + j] = d;
#pragma omp parallel for schedule(static)
        for (int i = j + 1; i < n; ++i) {
            double s = A[(size_t)i * n + j];
            const double* ri = &A[(size_t)i * n];
            const double* rj = &A[(size_t)j * n];
            for (int k = 0; k < j; ++k) s -= ri[k] * rj[k];
            A[(size_t)i * n + j] = s / d;
        }
    }
    return true;
}

// Solve (L L^T) x = b in place with the lower factor from cholesky().
void chol_solve(const std::vector<double>& Lf, int n, double* b) {
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        const double* ri = &Lf[(size_t)i * n];
        for (int k = 0; k < i; ++k) s -= ri[k] * b[k];
        b[i] = s / ri[i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= Lf[(size_t)k * n + i] * b[k];
        b[i] = s / Lf[(size_t)i * n + i];
    }
}

// Orthonormal Pbar_l^m(x), m in {0,1}, l = m..L at one node (x, sin t).
void pbar01(int m, int L, double x, double st, double* out /* index l */) {
    double prev = 0.0;
    double cur = (m == 0) ? std::sqrt(0.5) : -std::sqrt(0.75) * st;
    out[m] = cur;
    for (int l = m + 1; l <= L; ++l) {
        const double a = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
        double nxt;
        if (l == m + 1) {
            nxt = a * x * cur;
        } else {
            const double b = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) /
                                       (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
            nxt = a * (x * cur - b * prev);
        }
        prev = cur;
        cur = nxt;
        out[l] = cur;
    }
}

}  // namespace

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const int half = (n + 1) / 2;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < half; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) {
                // one more evaluation of the derivative at the converged node
                p0 = 1.0; p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                break;
            }
        }
        x[i] = z;                 // descending: x[0] is the largest node
        x[n - 1 - i] = -z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

std::string build_tables(int nside, int lmax, bool fp64, PlanTables& t) {
    const int ns = nside;
    const int p = 2 * ns;
    const int L = lmax;
    t.ns = ns; t.p = p; t.L = L; t.Q = 4 * ns + 1; t.npairs = 2 * ns;
    t.npix = 12LL * ns * ns;

    // ------------------------------------------------------------ rings
    const int np = t.npairs;
    t.nphi.resize(np); t.startN.resize(np); t.startS.resize(np); t.pow2.resize(np);
    t.logn.resize(np); t.fftL.resize(np); t.logL.resize(np);
    t.shOff.resize(np); t.chOff.resize(np); t.bhOff.resize(np);
    t.ch4Off.assign(np, 0); t.bh4Off.assign(np, 0);
    int64_t ch4N = 0, bh4N = 0;
    std::vector<double> phi0(np), theta(np);
    int64_t shN = 0, chN = 0, bhN = 0;
    int lmaxfft = 8 * ns;   // the latitude NUFFT grid
    t.smem_ring = 0;
    for (int i = 0; i < np; ++i) {
        const int j = i + 1;
        const int n = (j < ns) ? 4 * j : 4 * ns;
        const bool shifted = (j < ns) ? true : (j % 2 == 0);
        t.nphi[i] = n;
        t.startN[i] = (j < ns) ? 2 * j * (j - 1) : 2 * ns * (ns - 1) + (j - ns) * 4 * ns;
        t.startS[i] = (int)(t.npix - t.startN[i] - n);
        phi0[i] = shifted ? kPi / n : 0.0;
        t.shifted.push_back(shifted ? 1 : 0);
        theta[i] = ring_theta(j, ns);
        t.pow2[i] = is_pow2(n) ? 1 : 0;
        t.logn[i] = ilog2(n);
        int Lb = is_pow2(n) ? n : (1 << ilog2(2 * n - 1));
        t.fftL[i] = Lb;
        t.logL[i] = ilog2(Lb);
        t.smem_ring = std::max(t.smem_ring, Lb);
        lmaxfft = std::max(lmaxfft, Lb);
        t.shOff[i] = shN; shN += n / 2 + 1;
        t.chOff[i] = chN; t.bhOff[i] = bhN;
        if (!t.pow2[i]) {
            chN += n;
            bhN += Lb;
            t.ch4Off[i] = ch4N;
            t.bh4Off[i] = bh4N;
            ch4N += n / 4;
            bh4N += Lb / 4;
        }
    }
    t.chirp4.assign(2 * ch4N, 0.0);
    t.bhat4.assign(2 * bh4N, 0.0);
    t.Lmax = lmaxfft;
    t.shift.assign(2 * shN, 0.0);
    t.chirp.assign(2 * chN, 0.0);
    t.bhat.assign(2 * bhN, 0.0);
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < np; ++i) {
        const int n = t.nphi[i];
        const int h = n / 2;
        for (int m = 0; m <= h; ++m) {
            cd v;
            if (m < h) {
                v = std::polar(1.0 / n, -m * phi0[i]);
            } else if (h < p) {
                v = std::polar(0.5 / n, -m * phi0[i]);
            } else {   // equatorial Nyquist column p holds (c_{-p} + c_p) / 2
                v = cd(0.5 / n * std::cos(p * phi0[i]), 0.0);
            }
            t.shift[2 * (t.shOff[i] + m)] = v.real();
            t.shift[2 * (t.shOff[i] + m) + 1] = v.imag();
        }
        if (!t.pow2[i]) {
            const int Lb = t.fftL[i];
            std::vector<cd> b(Lb, cd(0.0, 0.0));
            for (int k = 0; k < n; ++k) {
                const long long r = ((long long)k * k) % (2LL * n);
                const double ang = kPi * (double)r / (double)n;
                t.chirp[2 * (t.chOff[i] + k)] = std::cos(ang);
                t.chirp[2 * (t.chOff[i] + k) + 1] = -std::sin(ang);
                b[k] = cd(std::cos(ang), std::sin(ang));
                if (k > 0) b[Lb - k] = b[k];
            }
            fft_host(b);
            for (int k = 0; k < Lb; ++k) {
                t.bhat[2 * (t.bhOff[i] + k)] = b[k].real() / Lb;
                t.bhat[2 * (t.bhOff[i] + k) + 1] = b[k].imag() / Lb;
            }
            // quarter-length subsequences: j = n / 4 points, convolution length Lb / 4 >= 2 j
            const int jq = n / 4, Lq = Lb / 4;
            std::vector<cd> bq(Lq, cd(0.0, 0.0));
            for (int u = 0; u < jq; ++u) {
                const long long r = ((long long)u * u) % (2LL * jq);
                const double ang = kPi * (double)r / (double)jq;
                t.chirp4[2 * (t.ch4Off[i] + u)] = std::cos(ang);
                t.chirp4[2 * (t.ch4Off[i] + u) + 1] = -std::sin(ang);
                bq[u] = cd(std::cos(ang), std::sin(ang));
                if (u > 0) bq[Lq - u] = bq[u];
            }
            fft_host(bq);
            for (int k = 0; k < Lq; ++k) {
                t.bhat4[2 * (t.bh4Off[i] + k)] = bq[k].real() / Lq;
                t.bhat4[2 * (t.bh4Off[i] + k) + 1] = bq[k].imag() / Lq;
            }
        }
    }
    t.twid.assign(2 * (size_t)t.Lmax, 0.0);   // Lmax complex: the full circle
    for (int k = 0; k < t.Lmax; ++k) {
        const double ang = -2.0 * kPi * (double)k / (double)t.Lmax;
        t.twid[2 * k] = std::cos(ang);
        t.twid[2 * k + 1] = std::sin(ang);
    }

    // ------------------------------------------------------------ pole fit
    {
        std::vector<double> xs, ys;
        t.poleN.clear(); t.poleS.clear();
        for (int i = 0; i < 3; ++i) {
            const int n = t.nphi[i];
            const double st = std::sin(theta[i]);
            for (int k = 0; k < n; ++k) {
                const double lam = phi0[i] + 2.0 * kPi * k / n;
                xs.push_back(st * std::cos(lam));
                ys.push_back(st * std::sin(lam));
                t.poleN.push_back(t.startN[i] + k);
                t.poleS.push_back(t.startS[i] + k);
            }
        }
        const int nP = (int)xs.size();
        std::vector<double> V((size_t)nP * 6);
        for (int k = 0; k < nP; ++k) {
            const double x = xs[k], y = ys[k];
            const double row[6] = {1.0, x, y, x * x, x * y, y * y};
            for (int c = 0; c < 6; ++c) V[(size_t)k * 6 + c] = row[c];
        }
        long double G[6][7];
        for (int a = 0; a < 6; ++a) {
            for (int b = 0; b < 6; ++b) {
                long double s = 0;
                for (int k = 0; k < nP; ++k) s += (long double)V[(size_t)k * 6 + a] * V[(size_t)k * 6 + b];
                G[a][b] = s;
            }
            G[a][6] = (a == 0) ? 1.0L : 0.0L;
        }
        for (int c = 0; c < 6; ++c) {   // Gauss-Jordan with partial pivoting
            int piv = c;
            for (int r = c + 1; r < 6; ++r) if (fabsl(G[r][c]) > fabsl(G[piv][c])) piv = r;
            if (fabsl(G[piv][c]) < 1e-300L) return "pole fit normal matrix is singular";
            for (int k = 0; k < 7; ++k) std::swap(G[c][k], G[piv][k]);
            for (int r = 0; r < 6; ++r) {
                if (r == c) continue;
                const long double f = G[r][c] / G[c][c];
                for (int k = c; k < 7; ++k) G[r][k] -= f * G[c][k];
            }
        }
        double g[6];
        for (int c = 0; c < 6; ++c) g[c] = (double)(G[c][6] / G[c][c]);
        t.polew.resize(nP);
        for (int k = 0; k < nP; ++k) {
            double s = 0.0;
            for (int c = 0; c < 6; ++c) s += g[c] * V[(size_t)k * 6 + c];
            t.polew[k] = s;
        }
    }

    // ------------------------------------------------------------ latitude nodes
    const int Q = t.Q;
    std::vector<double> th(Q);
    th[0] = 0.0;
    th[Q - 1] = kPi;
    for (int r = 1; r <= 2 * ns; ++r) th[r] = theta[r - 1];
    for (int r = 2 * ns + 1; r < Q - 1; ++r) th[r] = kPi - th[4 * ns - r];

    // ------------------------------------------------------------ ES NUFFT tables
    {
        const int M = 8 * ns;
        t.M = M;
        t.esw = fp64 ? HPX_ES_WIDTH_FP64 : HPX_ES_WIDTH_FP32;
        const double hgrid = 2.0 * kPi / M;
        const double alpha = t.esw * hgrid / 2.0;
        const double beta = 2.30 * t.esw;
        auto phi = [&](double z) { return (std::fabs(z) < 1.0) ? std::exp(beta * (std::sqrt(1.0 - z * z) - 1.0)) : 0.0; };
        std::vector<std::vector<std::pair<int, double>>> rows(M);
        auto add_node = [&](double tn, int code) {
            const int tlo = (int)std::ceil((tn - alpha) / hgrid);
            const int thi = (int)std::floor((tn + alpha) / hgrid);
            for (int tt = tlo; tt <= thi; ++tt) {
                const double z = (tt * hgrid - tn) / alpha;
                const double v = phi(z);
                if (v == 0.0) continue;
                const int tm = ((tt % M) + M) % M;
                rows[tm].push_back({code, v});
            }
        };
        for (int r = 0; r < Q; ++r) add_node(th[r], r);
        for (int r = 1; r < Q - 1; ++r) add_node(2.0 * kPi - th[r], r | (1 << 30));
        t.rowptr.assign(M + 1, 0);
        for (int i = 0; i < M; ++i) t.rowptr[i + 1] = t.rowptr[i] + (int)rows[i].size();
        t.ent.resize(t.rowptr[M]);
        t.entw.resize(t.rowptr[M]);
        for (int i = 0; i < M; ++i)
            for (size_t e = 0; e < rows[i].size(); ++e) {
                t.ent[t.rowptr[i] + e] = rows[i][e].first;
                t.entw[t.rowptr[i] + e] = rows[i][e].second;
            }
        // The same weights as a dense "first node + E weights" table: the DFS nodes
        // nu = 0 .. 8 Nside - 1 (nu <= 4 Nside: theta_nu; beyond: 2 pi - theta_{8 Nside - nu})
        // are sorted, so the nodes seen by one grid point form a cyclic run.
        {
            const int NN = 8 * ns;
            int E = 0;
            for (int i = 0; i < M; ++i) E = std::max(E, (int)rows[i].size());
            E = (E + 1) & ~1;
            t.spreadE = E;
            t.nstart.assign(M, 0);
            t.swts.assign((size_t)E * M, 0.0);
            for (int i = 0; i < M; ++i) {
                std::vector<std::pair<int, double>> nu;
                for (const auto& e : rows[i]) {
                    const int r = e.first & ((1 << 30) - 1);
                    nu.push_back({(e.first >> 30) ? NN - r : r, e.second});
                }
                if (nu.empty()) continue;
                std::sort(nu.begin(), nu.end());
                int start = nu.front().first;
                for (size_t k = 1; k < nu.size(); ++k)   // a wrap-around run starts after the gap
                    if (nu[k].first != nu[k - 1].first + 1) start = nu[k].first;
                t.nstart[i] = start;
                for (const auto& e : nu) {
                    const int off = ((e.first - start) % NN + NN) % NN;
                    if (off >= E) return "NUFFT spreading run is not contiguous";
                    t.swts[(size_t)off * M + i] = e.second;
                }
            }
        }
        // half grid with folded mirrors
        {
            const int H = M / 2;
            std::vector<std::vector<std::pair<int, std::pair<double, double>>>> hrow(H + 1);
            int E = 0;
            std::vector<int> rlo(H + 1, 0);
            for (int i = 0; i <= H; ++i) {
                int lo = Q, hi = -1;
                for (const auto& e : rows[i]) {
                    const int r = e.first & ((1 << 30) - 1);
                    lo = std::min(lo, r);
                    hi = std::max(hi, r);
                }
                if (hi < 0) { lo = 0; hi = 0; }
                rlo[i] = lo;
                E = std::max(E, hi - lo + 1);
            }
            t.spreadH = E;
            t.hstart.assign(H + 1, 0);
            t.hwts.assign((size_t)E * (H + 1) * 2, 0.0);
            for (int i = 0; i <= H; ++i) {
                const int st = std::min(rlo[i], Q - E);
                t.hstart[i] = st;
                for (const auto& e : rows[i]) {
                    const int r = e.first & ((1 << 30) - 1);
                    const bool mir = (e.first >> 30) != 0;
                    const size_t k = ((size_t)(r - st) * (H + 1) + i) * 2;
                    t.hwts[k] += e.second;
                    t.hwts[k + 1] += mir ? -e.second : e.second;
                }
            }
            for (int i = 1; i <= H; ++i)   // the spreading kernel relies on this
                if (t.hstart[i] < t.hstart[i - 1]) return "half-grid spreading starts are not monotone";
            int rows32 = 0;
            for (int t0 = 0; t0 <= H; t0 += 32)
                rows32 = std::max(rows32, t.hstart[std::min(t0 + 31, H)] + E - t.hstart[t0]);
            t.spreadRows = rows32;
            // the same weights grouped by latitude node: node r sees the half-grid
            // points tstart[r] .. tstart[r] + En - 1 (a contiguous run, since the
            // first node of a grid point never decreases) with weights
            // hwn[e][r][2] = hwts of that (grid point, node), zero outside its run
            {
                std::vector<int> tlo(Q, H + 1), thi(Q, -1);
                for (int i = 0; i <= H; ++i)
                    for (int e = 0; e < E; ++e) {
                        const size_t k = ((size_t)e * (H + 1) + i) * 2;
                        if (t.hwts[k] == 0.0 && t.hwts[k + 1] == 0.0) continue;   // outside the kernel's support
                        const int r = t.hstart[i] + e;
                        tlo[r] = std::min(tlo[r], i);
                        thi[r] = std::max(thi[r], i);
                    }
                int En = 1;
                for (int r = 0; r < Q; ++r)
                    if (thi[r] >= tlo[r]) En = std::max(En, thi[r] - tlo[r] + 1);
                t.interpE = En;
                t.tstart.assign(Q, 0);
                t.hwn.assign((size_t)En * Q * 2, 0.0);
                for (int r = 0; r < Q; ++r) {
                    const int st = (thi[r] < tlo[r]) ? 0 : std::min(tlo[r], H + 1 - En);
                    t.tstart[r] = st;
                    for (int i = std::max(st, 0); i < st + En && i <= H; ++i) {
                        const int e = r - t.hstart[i];
                        if (e < 0 || e >= E) continue;
                        const size_t k = ((size_t)e * (H + 1) + i) * 2;
                        const size_t q = ((size_t)(i - st) * Q + r) * 2;
                        t.hwn[q] = t.hwts[k];
                        t.hwn[q + 1] = t.hwts[k + 1];
                    }
                }
                int rows32 = 0;   // grid points seen by 32 consecutive nodes (at most)
                for (int r0 = 0; r0 < Q; r0 += 32)
                    rows32 = std::max(rows32, t.tstart[std::min(r0 + 31, Q - 1)] + En - t.tstart[r0]);
                t.interpRows = rows32;
                t.interpD = 0;   // spread of the run starts over 4 consecutive nodes (from r = 0, 4, 8, ..)
                for (int r0 = 0; r0 < Q; r0 += 4)
                    t.interpD = std::max(t.interpD, t.tstart[std::min(r0 + 3, Q - 1)] - t.tstart[r0]);
            }

            t.spreadD = 0;
            for (int t0 = 0; t0 <= H; t0 += 4) t.spreadD = std::max(t.spreadD, t.hstart[std::min(t0 + 3, H)] - t.hstart[t0]);
        }
        // the same entries grouped by latitude node (for the transposed NUFFT)
        std::vector<std::vector<std::pair<int, double>>> byNode(Q);
        for (int i = 0; i < M; ++i)
            for (const auto& e : rows[i]) {
                const int r = e.first & ((1 << 30) - 1);
                const int mir = e.first >> 30;
                byNode[r].push_back({i | (mir << 30), e.second});
            }
        t.nrowptr.assign(Q + 1, 0);
        for (int r = 0; r < Q; ++r) t.nrowptr[r + 1] = t.nrowptr[r] + (int)byNode[r].size();
        t.nent.resize(t.nrowptr[Q]);
        t.nentw.resize(t.nrowptr[Q]);
        for (int r = 0; r < Q; ++r)
            for (size_t e = 0; e < byNode[r].size(); ++e) {
                t.nent[t.nrowptr[r] + e] = byNode[r][e].first;
                t.nentw[t.nrowptr[r] + e] = byNode[r][e].second;
            }
        std::vector<double> zg, wz;
        gauss_legendre(512, zg, wz);
        t.dec.resize(p + 1);
        for (int j = 0; j <= p; ++j) {
            double s = 0.0;
            for (size_t g = 0; g < zg.size(); ++g) s += wz[g] * phi(zg[g]) * std::cos(j * alpha * zg[g]);
            t.dec[j] = hgrid / (alpha * s);
        }
    }

    // ------------------------------------------------------------ latitude LS operator
    {
        const int P2 = p / 2 + 1;
        t.P2 = P2;
        t.D.assign((size_t)4 * P2 * P2, 0.0);
        t.C.assign((size_t)4 * P2 * P2, 0.0);
        std::vector<double> tc(2 * p + 1), ts(2 * p + 1);
        for (int k = 0; k <= 2 * p; ++k) {
            double sc = 0.0, ss = 0.0;
            for (int r = 0; r < Q; ++r) {
                const double c = std::cos(k * th[r]);
                const double wr = (r == 0 || r == Q - 1) ? 1.0 : 2.0;
                sc += wr * c;
                if (r > 0 && r < Q - 1) ss += c;
            }
            tc[k] = sc;
            ts[k] = ss;
        }
        t.tc = tc;
        t.ts = ts;
        const int G = p + 2;   // exact for the polynomial integrands of degree <= 2p
        std::vector<double> xg, wg;
        gauss_legendre(G, xg, wg);
        const int Gh = G / 2;  // nodes with x > 0 (G even)
        // Pbar_l^{0,1} and cos/sin(j theta) at the positive half of the nodes
        std::vector<double> P0((size_t)(L + 1) * Gh, 0.0), P1((size_t)(L + 1) * Gh, 0.0);
        std::vector<double> CJ((size_t)(p + 1) * Gh), SJ((size_t)(p + 1) * Gh);
#pragma omp parallel for schedule(static)
        for (int g = 0; g < Gh; ++g) {
            const double x = xg[g];
            const double st = std::sqrt((1.0 - x) * (1.0 + x));
            const double tg = std::acos(x);
            std::vector<double> buf(L + 1);
            pbar01(0, L, x, st, buf.data());
            for (int l = 0; l <= L; ++l) P0[(size_t)l * Gh + g] = buf[l];
            if (L >= 1) {
                pbar01(1, L, x, st, buf.data());
                for (int l = 1; l <= L; ++l) P1[(size_t)l * Gh + g] = buf[l];
            }
            for (int j = 0; j <= p; ++j) {
                CJ[(size_t)j * Gh + g] = std::cos(j * tg);
                SJ[(size_t)j * Gh + g] = std::sin(j * tg);
            }
        }
        const double s2pi = std::sqrt(2.0 * kPi);
        for (int mpar = 0; mpar < 2; ++mpar) {
            for (int par = 0; par < 2; ++par) {
                std::vector<int> js, ls;
                for (int j = (mpar ? 1 : 0); j <= p; ++j) if ((j & 1) == par) js.push_back(j);
                for (int l = (mpar ? 1 : 0); l <= L; ++l) if ((l & 1) == par) ls.push_back(l);
                const int nj = (int)js.size(), nl = (int)ls.size();
                if (nj == 0 || nl == 0) continue;
                std::vector<double> T((size_t)nj * nj);
                for (int a = 0; a < nj; ++a)
                    for (int b = 0; b < nj; ++b) {
                        const int ja = js[a], jb = js[b];
                        T[(size_t)a * nj + b] = mpar == 0
                            ? 0.5 * (tc[std::abs(ja - jb)] + tc[ja + jb])
                            : 0.5 * (ts[std::abs(ja - jb)] - ts[ja + jb]);
                    }
                if (!cholesky(T, nj)) return "latitude Gram matrix is not positive definite";
                const std::vector<double>& PL = mpar ? P1 : P0;
                const std::vector<double>& BJ = mpar ? SJ : CJ;
#pragma omp parallel for schedule(dynamic, 8)
                for (int a = 0; a < nl; ++a) {
                    const int l = ls[a];
                    std::vector<double> row(nj);
                    const double* pl = &PL[(size_t)l * Gh];
                    for (int b = 0; b < nj; ++b) {
                        const double* bj = &BJ[(size_t)js[b] * Gh];
                        double s = 0.0;
                        for (int g = 0; g < Gh; ++g) s += wg[g] * pl[g] * bj[g];
                        row[b] = 2.0 * s;   // the integrand is even in x
                    }
                    const int q = l >> 1;
                    for (int b = 0; b < nj; ++b)
                        t.C[(((size_t)mpar * 2 + par) * P2 + q) * P2 + (js[b] >> 1)] = s2pi * row[b];
                    chol_solve(T, nj, row.data());   // row <- T^{-1} row (T symmetric)
                    for (int b = 0; b < nj; ++b) {
                        const int k = js[b] >> 1;
                        t.D[(((size_t)mpar * 2 + par) * P2 + q) * P2 + k] = s2pi * row[b];
                    }
                }
            }
        }
    }

    // ------------------------------------------------------------ Givens angles
    {
        t.angOff.assign((size_t)(L + 1) * 2 + 2, 0);
        int64_t off = 0;
        for (int mp = 0; mp <= L; ++mp)
            for (int c = 0; c < 2; ++c) {
                t.angOff[(size_t)mp * 2 + c] = off;
                off += chain_len(mp + 2, c, L);
            }
        t.angOff[(size_t)(L + 1) * 2] = off;
        t.ang.assign(2 * off, 0.0);
#pragma omp parallel for schedule(dynamic, 4)
        for (int mp = 0; mp <= L; ++mp) {
            for (int c = 0; c < 2; ++c) {
                const int n = chain_len(mp + 2, c, L);
                if (n <= 0) continue;
                auto A = [&](int l) -> double {
                    if (l < mp) return 0.0;
                    const double num = (double)(l + 1) * (l + 1) - (double)mp * mp;
                    return std::sqrt(std::max(num, 0.0) / ((2.0 * l + 1.0) * (2.0 * l + 3.0)));
                };
                auto li = [&](int i) { return mp + c + 2 * i; };
                auto Jd = [&](int i) { const double a1 = A(li(i)), a0 = A(li(i) - 1); return 1.0 - a1 * a1 - a0 * a0; };
                auto Jo = [&](int i) { return -A(li(i)) * A(li(i) + 1); };   // J_{i+1,i}
                double a = Jd(0), cprev = 1.0;
                const int64_t o = t.angOff[(size_t)mp * 2 + c];
                for (int k = 0; k < n; ++k) {
                    const double b = Jo(k);
                    const double r = std::hypot(a, b);
                    const double cc = a / r, ss = b / r;
                    t.ang[2 * (o + k)] = cc;
                    t.ang[2 * (o + k) + 1] = ss;
                    a = -ss * (cprev * Jo(k)) + cc * Jd(k + 1);
                    cprev = cc;
                }
            }
        }
        // skewed copy for the register wavefront (rows of 32 (cos, sin) pairs)
        const int nq = (L / 2 + 31) / 32 + 1;
        t.nq = nq;
        t.skOff.assign((size_t)4 * nq + 1, 0);
        int64_t rows = 0;
        for (int m0 = 0; m0 < 2; ++m0)
            for (int c = 0; c < 2; ++c)
                for (int q = 0; q < nq; ++q) {
                    t.skOff[(size_t)(m0 * 2 + c) * nq + q] = rows;
                    const int n0 = chain_len(m0 + 64 * q, c, L);
                    rows += (n0 > 0) ? n0 + 62 : 0;
                }
        t.skOff[(size_t)4 * nq] = rows;
        t.skew.assign((size_t)rows * 64, 0.0);
        for (int64_t r = 0; r < rows; ++r)
            for (int k = 0; k < 32; ++k) t.skew[(size_t)r * 64 + 2 * k] = 1.0;
#pragma omp parallel for collapse(3) schedule(dynamic, 1)
        for (int m0 = 0; m0 < 2; ++m0)
            for (int c = 0; c < 2; ++c)
                for (int q = 0; q < nq; ++q) {
                    const int n0 = chain_len(m0 + 64 * q, c, L);
                    if (n0 <= 0) continue;
                    const int64_t base = t.skOff[(size_t)(m0 * 2 + c) * nq + q];
                    for (int k = 0; k < 32; ++k) {
                        const int mp = m0 + 2 * (32 * q + k);   // order entering stage 32q+k
                        if (mp + 2 > L + 1) continue;
                        const int nrot = chain_len(mp + 2, c, L);
                        const int64_t o = t.angOff[(size_t)mp * 2 + c];
                        for (int i = 1; i <= nrot; ++i) {
                            const int64_t row = base + i + 2 * k;
                            if (row >= base + n0 + 62) break;
                            t.skew[(size_t)row * 64 + 2 * k] = t.ang[2 * (o + i - 1)];
                            t.skew[(size_t)row * 64 + 2 * k + 1] = t.ang[2 * (o + i - 1) + 1];
                        }
                    }
                }
        // reverse (transposed) sweeps: stage k of block q undoes forward stage 32q+31-k
        t.skewT.assign((size_t)rows * 64, 0.0);
#pragma omp parallel for collapse(3) schedule(dynamic, 1)
        for (int m0 = 0; m0 < 2; ++m0)
            for (int c = 0; c < 2; ++c)
                for (int q = 0; q < nq; ++q) {
                    const int n0 = chain_len(m0 + 64 * q, c, L);
                    if (n0 <= 0) continue;
                    const int64_t base = t.skOff[(size_t)(m0 * 2 + c) * nq + q];
                    const int64_t nrows = n0 + 62;
                    for (int k = 0; k < 32; ++k) {
                        const int s = 32 * q + 31 - k;
                        const int mp = m0 + 2 * s;
                        const int ns = (mp + 2 <= L + 1) ? chain_len(mp + 2, c, L) : 0;
                        const int64_t o = (mp <= L) ? t.angOff[(size_t)mp * 2 + c] : 0;
                        for (int64_t tt = 0; tt < nrows; ++tt) {
                            const int64_t i = ns + k - tt;
                            double cs = 0.0, sn = 0.0;
                            if (i >= 1 && i <= ns) {
                                cs = t.ang[2 * (o + i - 1)];
                                sn = t.ang[2 * (o + i - 1) + 1];
                            } else if (i == 0) {
                                cs = 1.0;
                            }
                            t.skewT[(size_t)(base + tt) * 64 + 2 * k] = cs;
                            t.skewT[(size_t)(base + tt) * 64 + 2 * k + 1] = sn;
                        }
                    }
                }
    }
    return "";
}

void build_synthesis_table(const PlanTables& t, std::vector<double>& Es) {
    const int p = t.p, L = t.L, P2 = t.P2;
    Es.assign((size_t)4 * P2 * P2, 0.0);
    // midpoint rule in t on [0, pi] with N points integrates cos(k t) exactly for
    // 0 < k < 2N; the products Pbar_l B_j have degree <= L + p < 2N
    const int N = p + 2;
    std::vector<double> tn(N);
    for (int n = 0; n < N; ++n) tn[n] = kPi * (n + 0.5) / N;
    const double inv = 1.0 / std::sqrt(2.0 * kPi);
    for (int m0 = 0; m0 < 2; ++m0) {
        if (L < m0) continue;
        std::vector<double> PL((size_t)(L + 1) * N, 0.0);   // Pbar_l^{m0}(cos t_n)
#pragma omp parallel for schedule(static)
        for (int n = 0; n < N; ++n) {
            std::vector<double> buf(L + 1);
            pbar01(m0, L, std::cos(tn[n]), std::sin(tn[n]), buf.data());
            for (int l = m0; l <= L; ++l) PL[(size_t)l * N + n] = buf[l];
        }
#pragma omp parallel for schedule(dynamic, 4)
        for (int j = m0; j <= p; ++j) {
            std::vector<double> bj(N);
            for (int n = 0; n < N; ++n) bj[n] = m0 ? std::sin(j * tn[n]) : std::cos(j * tn[n]);
            // E_jl = 2 / (pi (1 + [j = 0])) * integral_0^pi Pbar_l(cos t) B_j(t) dt
            const double scale = (2.0 / kPi) / (j == 0 ? 2.0 : 1.0) * (kPi / N);
            const int par = j & 1;
            for (int l = (m0 > par ? m0 + 1 : par); l <= L; l += 2) {
                if (l < m0) continue;
                const double* pl = &PL[(size_t)l * N];
                double s = 0.0;
                for (int n = 0; n < N; ++n) s += pl[n] * bj[n];
                Es[(((size_t)m0 * 2 + par) * P2 + (l >> 1)) * P2 + (j >> 1)] = scale * s * inv;
            }
        }
    }
}

void build_cg_tables(const PlanTables& t, int& N, std::vector<double>& H, int k0[4], int n[4]) {
    const int P2 = t.P2;
    int nmax = 0;
    for (int blk = 0; blk < 4; ++blk) {
        const int mpar = blk >> 1, par = blk & 1;
        k0[blk] = (mpar == 1 && par == 0) ? 1 : 0;
        const int k1 = par == 0 ? P2 - 1 : P2 - 2;
        n[blk] = std::max(0, k1 - k0[blk] + 1);
        nmax = std::max(nmax, n[blk]);
    }
    N = 1;
    while (N < 3 * nmax - 2) N <<= 1;
    H.assign((size_t)4 * 2 * N * 2, 0.0);
    for (int blk = 0; blk < 4; ++blk) {
        const int mpar = blk >> 1, par = blk & 1, nn = n[blk];
        if (nn == 0) continue;
        const std::vector<double>& tt = mpar ? t.ts : t.tc;
        const double sg = mpar ? -1.0 : 1.0;
        std::vector<double> cvec(N, 0.0), gvec(N, 0.0);
        for (int d = 0; d < nn; ++d) {
            cvec[d] = 0.5 * tt[2 * d];
            if (d > 0) cvec[N - d] = 0.5 * tt[2 * d];
        }
        for (int e = 0; e <= 2 * nn - 2; ++e) gvec[e] = sg * 0.5 * tt[2 * e + 4 * k0[blk] + 2 * par];
        double* Hc = &H[((size_t)blk * 2 + 0) * N * 2];
        double* Hg = &H[((size_t)blk * 2 + 1) * N * 2];
#pragma omp parallel for schedule(static)
        for (int k = 0; k < N; ++k) {
            double cr = 0, ci = 0, gr = 0, gi = 0;
            for (int i = 0; i < N; ++i) {
                if (cvec[i] == 0.0 && gvec[i] == 0.0) continue;
                const double a = -2.0 * kPi * (double)(((int64_t)k * i) % N) / N;
                const double cs = std::cos(a), sn = std::sin(a);
                cr += cvec[i] * cs; ci += cvec[i] * sn;
                gr += gvec[i] * cs; gi += gvec[i] * sn;
            }
            Hc[2 * k] = cr / N; Hc[2 * k + 1] = ci / N;
            Hg[2 * k] = gr / N; Hg[2 * k + 1] = gi / N;
        }
    }
}

}  // namespace hpx
