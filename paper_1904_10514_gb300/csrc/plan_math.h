// Host-side (FP64) set-up of the HP2SPH plan tables.  Everything here runs once
// per plan; the per-map work is in the CUDA kernels.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace hpx {

struct PlanTables {
    int ns = 0;      // N_side
    int p = 0;       // 2 N_side: longitude/latitude half-bandwidth
    int L = 0;       // lmax <= p
    int Q = 0;       // 4 N_side + 1 latitude nodes on [0, pi] (poles included)
    int npairs = 0;  // 2 N_side north/south ring pairs (the equator pairs with itself)
    int64_t npix = 0;

    // ---- Step 1 (Sec. 3.1): per ring pair i (north ring i, south ring 4Ns-2-i)
    std::vector<int> nphi, startN, startS, pow2, logn, fftL, logL;
    std::vector<int> shifted;    // 1: first pixel at longitude pi / nphi, 0: at 0
    std::vector<int64_t> shOff, chOff, bhOff;
    std::vector<double> shift;   // complex: (1/nphi) e^{-i m phi0}, Nyquist split folded in
    std::vector<double> chirp;   // complex: e^{-i pi k^2 / nphi} (Bluestein rings)
    std::vector<double> bhat;    // complex: FFT_L of the conjugate chirp, divided by L
    // the same for the quarter-length subsequences z[4u + s] of a Bluestein ring
    // (nphi = 4j: DFT_nphi from four DFT_j, each by Bluestein with L / 4 points)
    std::vector<int64_t> ch4Off, bh4Off;
    std::vector<double> chirp4;  // complex: e^{-i pi u^2 / j}, u < j
    std::vector<double> bhat4;   // complex: FFT_{L/4} of the conjugate chirp, divided by L / 4
    int Lmax = 0;                // twiddle table covers FFT lengths up to Lmax
    std::vector<double> twid;    // complex: e^{-2 pi i k / Lmax}, k < Lmax/2
    int smem_ring = 0;           // largest in-CTA FFT length of step 1

    // ---- pole values (Sec. 3.2.1)
    std::vector<double> polew;   // weights over the pixels of the 3 rings nearest a pole
    std::vector<int> poleN, poleS;  // pixel indices (north / mirrored south)

    // ---- DFS + type-1 NUFFT in latitude (Sec. 3.2.1-3.2.2)
    int M = 0;                   // fine grid size 8 N_side
    int esw = 0;                 // exponential-of-semicircle kernel width (grid cells)
    std::vector<int> rowptr;     // CSR over fine-grid points
    std::vector<int> ent;        // node index r | (mirrored << 30)
    std::vector<double> entw;    // kernel weight
    std::vector<double> dec;     // h / Phi(j), j = 0..p (deconvolution)
    int spreadE = 0;             // weights per grid point in the dense spreading table
    std::vector<int> nstart;     // first DFS node seen by grid point t (cyclic run of spreadE)
    std::vector<double> swts;    // [spreadE][M] weights, zero past the end of a run
    // The same spreading on the half grid t = 0..M/2 with the mirrored nodes
    // folded in (the grid values obey u[M - t] = (-1)^m u[t]): grid point t sees
    // the latitude nodes r = hstart[t] .. hstart[t] + spreadH - 1 with weights
    // hwts[e][t] = (w(even m), w(odd m)); spreadRows bounds the nodes seen by 32
    // consecutive grid points.
    int spreadH = 0, spreadRows = 0;
    int spreadD = 0;             // max of hstart[t + 3] - hstart[t] over t = 0, 4, 8, ..
    std::vector<int> hstart;
    std::vector<double> hwts;    // [spreadH][M/2 + 1][2]
    // The transpose (interpolation from the half grid to the latitude nodes):
    // node r takes the grid points tstart[r] .. tstart[r] + interpE - 1 with
    // weights hwn[e][r][2] (even m, odd m); interpRows bounds the grid points
    // that 32 consecutive nodes see.
    int interpE = 0, interpRows = 0, interpD = 0;
    std::vector<int> tstart;
    std::vector<double> hwn;     // [interpE][Q][2]

    // ---- latitude least squares + Chebyshev -> order-0/1 Legendre (Sec. 3.2.2, 3.3)
    int P2 = 0;                  // p/2 + 1
    std::vector<double> D;       // [mpar][par][P2][P2], rows q -> l = 2q+par, cols k -> j = 2k+par
    // The two factors of D = C T^{-1}: C = sqrt(2 pi) <Pbar_l, B_j> (the change of
    // basis, same layout as D) and the normal-equation matrix T of each (mpar, par)
    // block, T_ab = (tt[|j_a - j_b|] +- tt[j_a + j_b]) / 2 with tt = tc (cosine,
    // +) or ts (sine, -), j = 0..2p (the conjugate-gradient form, HPX_FLAG_CG)
    std::vector<double> C, tc, ts;

    // ---- Givens rotations of the order m' -> m'+2 connection (Sec. 3.3)
    std::vector<int64_t> angOff; // [(L+1) * 2]: offset of (m', chain c)
    std::vector<double> ang;     // (cos, sin) pairs
    // The same angles re-laid for the register wavefront of the sweep kernel:
    // for start parity m0, chain c and block q of 32 stages (stages 32q..32q+31,
    // orders m' = m0 + 2 s), row t, column k holds the angle that stage 32q+k
    // applies at time step t (rotation index t - 2k), or (1, 0) where that stage
    // is idle.  skOff[(m0 * 2 + c) * nq + q] = first row; each row = 32 pairs.
    int nq = 0;
    std::vector<int64_t> skOff;
    std::vector<double> skew;
    // Transposed sweeps (the adjoint): reverse stage k of block q undoes forward
    // stage 32q+31-k; row t, column k holds its angle at rotation index
    // i = n_s + k - t (n_s = rotations of that stage), (1, 0) at i = 0 (emit the
    // carry), (0, 0) elsewhere (clear the carry / idle).  Same offsets as skOff.
    std::vector<double> skewT;

    // ---- transpose of the NUFFT spreading: CSR over latitude nodes
    std::vector<int> nrowptr;    // [Q + 1]
    std::vector<int> nent;       // grid point t | (mirrored << 30)
    std::vector<double> nentw;
};

// Build all tables; returns an empty string on success or a message.
std::string build_tables(int nside, int lmax, bool fp64, PlanTables& t);

// Spherical-harmonic synthesis (the inverse direction of Sec. 3.3): the exact
// expansion of the order-0/1 normalised Legendre functions in the latitude
// Fourier basis, Pbar_l^{m0}(cos t) = sum_j E_{jl} cos(j t) (m0 = 0) or
// sin(j t) (m0 = 1), j = l mod 2, scaled by 1/sqrt(2 pi) (Appendix A:
// Y_l^m = Pbar_l^m e^{i m phi} / sqrt(2 pi)).  Laid out like D:
// Es[m0][par][q][k] = E_{2k+par, 2q+par} / sqrt(2 pi).
void build_synthesis_table(const PlanTables& t, std::vector<double>& Es);

// Conjugate-gradient form of the latitude least squares (Sec. 3.2.2: CG on the
// normal equations, matrix-vector products by FFT).  For block (mpar, par) the
// unknowns are the modes k = k0 .. k0 + n - 1 (j = 2k + par); T x is
// IFFT_N(Hc . X + Hg . X(-k)) restricted to the first n entries, X = FFT_N(x):
// Hc holds the circulant embedding of the Toeplitz part, Hg the Hankel part,
// both divided by N (N = the power of two >= 3n - 2).  Layout H[blk][2][N]
// complex (blk = 2 mpar + par); k0[blk], n[blk].
void build_cg_tables(const PlanTables& t, int& N, std::vector<double>& H, int k0[4], int n[4]);

// Gauss-Legendre nodes/weights on [-1, 1] (Newton on the Legendre recurrence).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// Chain length of order m', parity chain c (degrees m'+c+2i <= L).
#if defined(__CUDACC__)
__host__ __device__
#endif
inline int chain_len(int mp, int c, int L) { return (L >= mp + c) ? (L - mp - c) / 2 + 1 : 0; }

}  // namespace hpx
