/*
 * FP64 reference sampler for the lattice path-integral Coulomb method
 * (Sugihara, Higo & Nakamura, "Local Representation of N-body Coulomb Energy
 * with Path Integrals", JPSJ 2014).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the product library never does.  It shares
 * no code, header, table or helper with the CUDA sources.
 *
 * Everything here is deliberately plain: one site at a time, natural
 * x-fastest field order phi[x + Lx*(y + Ly*z)], double precision throughout,
 * one Philox call per site (the GPU path shares one call between four sites).
 *
 * What each function follows:
 *   orc_philox4x32_10  Philox4x32-10 counter-based generator, as published by
 *                      Salmon, Moraes, Dror & Shaw (SC'11): 10 rounds of two
 *                      32x32->64 multiplies with a Weyl key schedule.
 *   orc_erfcinv        inverse of the complementary error function, Newton's
 *                      method on erfc() started from Winitzki's closed-form
 *                      approximation of erf^-1 (2008).  Needed by Eq. (phi).
 *   orc_halfsweep      heatbath update Eq. (phi) (inversion of Eq. (hb1)) for
 *                      every site of one checkerboard colour, with Dirichlet
 *                      phi=0 outside the box (the paper's open-boundary
 *                      modification), or the over-relaxation reflection
 *                      phi -> S/3 - phi about the same conditional mean.
 *   orc_measure        one term of Eq. (nsum2): Q = sum q_i phi_{n_i},
 *                      P = sum (q_i phi_{n_i})^2, e = Q^2 - P.
 *   orc_run            thermalisation / measured compound sweeps.
 *
 * Readings of the paper fixed here (the CUDA path takes the same ones):
 *   - H_L counts each nearest-neighbour pair once, including the links to the
 *     phi=0 ghost layer, so the conditional law of phi_n is N(S_n/6, 1/6)
 *     (the 1/sqrt(3) in front of erfc^-1 in Eq. (phi) is sqrt(2)/sqrt(6)).
 *   - The uniform r of Eq. (hb1) is r = (w + 1/2) 2^-32 for a 32-bit Philox
 *     word w, so 0 < r < 1 and Eq. (phi) is finite.  erfc^-1(2r) is evaluated
 *     as -erfc^-1(2 - 2r) when 2r > 1 (an identity of erfc) to keep precision.
 *   - Sites are visited colour by colour (red = (x+y+z) even first) rather
 *     than in one sequential sweep; every site of one colour depends only on
 *     the other colour, so the order within a colour does not matter.
 *   - The Philox counter of a heatbath update of site (x,y,z), colour c,
 *     during pass number `pass` of chain `chain` is
 *       (qid, pass, chain, c),  qid = (z*Ly + y)*Wq + (x>>3),  Wq = ceil(Lx/8),
 *     the key is (seed mod 2^32, seed div 2^32), and the site takes output
 *     word ((x>>1) & 3).  Over-relaxation passes draw nothing but still count
 *     in `pass`.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                       */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u; /* Weyl key schedule */
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------ */
/* erfc^-1                                                             */
/* ------------------------------------------------------------------ */
/* y >= 0 with erfc(y) = u, for 0 < u <= 1. */
static double erfcinv_unit(double u)
{
    if (u >= 1.0) return 0.0;
    /* Winitzki: erf^-1(z) ~ sqrt( sqrt(t^2 - l/a) - t ), t = 2/(pi a) + l/2,
     * l = ln(1 - z^2), a = 0.147.  Here z = 1 - u, so 1 - z^2 = u (2 - u). */
    const double a = 0.147;
    double l = log(u * (2.0 - u));
    double t = 2.0 / (ORC_PI * a) + 0.5 * l;
    double y = sqrt(sqrt(t * t - l / a) - t);
    /* Newton on f(y) = erfc(y) - u, f'(y) = -(2/sqrt(pi)) exp(-y^2). */
    for (int it = 0; it < 6; ++it) {
        double f = erfc(y) - u;
        double fp = -2.0 / sqrt(ORC_PI) * exp(-y * y);
        y -= f / fp;
    }
    return y;
}

/* erfc^-1(v) for 0 < v < 2. */
double orc_erfcinv(double v)
{
    if (v <= 1.0) return erfcinv_unit(v);
    return -erfcinv_unit(2.0 - v);
}

/* ------------------------------------------------------------------ */
/* Sweeps                                                              */
/* ------------------------------------------------------------------ */
static double neighbour_sum(const double *phi, int Lx, int Ly, int Lz, int x, int y, int z)
{
    /* Sum over the six nearest neighbours; sites outside the box are phi=0. */
    double s = 0.0;
    if (x > 0)      s += phi[(x - 1) + (size_t)Lx * (y + (size_t)Ly * z)];
    if (x < Lx - 1) s += phi[(x + 1) + (size_t)Lx * (y + (size_t)Ly * z)];
    if (y > 0)      s += phi[x + (size_t)Lx * ((y - 1) + (size_t)Ly * z)];
    if (y < Ly - 1) s += phi[x + (size_t)Lx * ((y + 1) + (size_t)Ly * z)];
    if (z > 0)      s += phi[x + (size_t)Lx * (y + (size_t)Ly * (z - 1))];
    if (z < Lz - 1) s += phi[x + (size_t)Lx * (y + (size_t)Ly * (z + 1))];
    return s;
}

/* The 32-bit word that the heatbath update of (x,y,z) consumes. */
uint32_t orc_site_word(int Lx, int Ly, int x, int y, int z, int colour,
                       uint64_t seed, uint32_t chain, uint32_t pass)
{
    uint32_t Wq = (uint32_t)((Lx + 7) / 8);
    uint32_t qid = ((uint32_t)z * (uint32_t)Ly + (uint32_t)y) * Wq + (uint32_t)(x >> 3);
    uint32_t ctr[4] = { qid, pass, chain, (uint32_t)colour };
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    return w[(x >> 1) & 3];
}

/* The deviate -erfc^-1(2r)/sqrt(3) that Eq. (phi) adds to S/6, for word w. */
double orc_heatbath_noise(uint32_t w)
{
    double r = ((double)w + 0.5) * 0x1p-32;
    return -orc_erfcinv(2.0 * r) / sqrt(3.0);
}

/* One half-sweep over colour `colour` (0 = red, (x+y+z) even).
 * heatbath != 0: Eq. (phi); heatbath == 0: over-relaxation.
 * noise_scale multiplies the random term (1 for the sampler; 0 turns the
 * heatbath into a red/black Gauss-Seidel step, used by the oracle's tests). */
void orc_halfsweep(double *phi, int Lx, int Ly, int Lz, int colour, int heatbath,
                   uint64_t seed, uint32_t chain, uint32_t pass, double noise_scale)
{
#pragma omp parallel for schedule(static)
    for (int z = 0; z < Lz; ++z) {
        for (int y = 0; y < Ly; ++y) {
            for (int x = 0; x < Lx; ++x) {
                if (((x + y + z) & 1) != colour) continue;
                size_t n = x + (size_t)Lx * (y + (size_t)Ly * z);
                double S = neighbour_sum(phi, Lx, Ly, Lz, x, y, z);
                if (heatbath) {
                    uint32_t w = orc_site_word(Lx, Ly, x, y, z, colour, seed, chain, pass);
                    phi[n] = S / 6.0 + noise_scale * orc_heatbath_noise(w);
                } else {
                    phi[n] = S / 3.0 - phi[n];
                }
            }
        }
    }
}

/* One pass = red half-sweep then black half-sweep. */
void orc_pass(double *phi, int Lx, int Ly, int Lz, int heatbath,
              uint64_t seed, uint32_t chain, uint32_t pass, double noise_scale)
{
    orc_halfsweep(phi, Lx, Ly, Lz, 0, heatbath, seed, chain, pass, noise_scale);
    orc_halfsweep(phi, Lx, Ly, Lz, 1, heatbath, seed, chain, pass, noise_scale);
}

/* ------------------------------------------------------------------ */
/* Estimator, Eq. (nsum2)                                              */
/* ------------------------------------------------------------------ */
void orc_measure(const double *phi, const int64_t *site, const double *q, int64_t n,
                 double out[3])
{
    double Q = 0.0, P = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double t = q[i] * phi[site[i]];
        Q += t;
        P += t * t;
    }
    out[0] = Q;
    out[1] = P;
    out[2] = Q * Q - P;
}

/* H_L = 1/2 sum over nearest-neighbour pairs (phi_m - phi_n)^2, every pair
 * once, including the pairs (boundary site, ghost site) with ghost phi = 0. */
double orc_action(const double *phi, int Lx, int Ly, int Lz)
{
    double h = 0.0;
    for (int z = -1; z < Lz; ++z)
        for (int y = -1; y < Ly; ++y)
            for (int x = -1; x < Lx; ++x) {
                /* links from (x,y,z) to (x+1,y,z), (x,y+1,z), (x,y,z+1) */
                int in0 = x >= 0 && y >= 0 && z >= 0;
                double p0 = in0 ? phi[x + (size_t)Lx * (y + (size_t)Ly * z)] : 0.0;
                if (y >= 0 && z >= 0) {
                    double p1 = (x + 1 < Lx) ? phi[(x + 1) + (size_t)Lx * (y + (size_t)Ly * z)] : 0.0;
                    if (in0 || x + 1 < Lx) h += 0.5 * (p1 - p0) * (p1 - p0);
                }
                if (x >= 0 && z >= 0) {
                    double p1 = (y + 1 < Ly) ? phi[x + (size_t)Lx * ((y + 1) + (size_t)Ly * z)] : 0.0;
                    if (in0 || y + 1 < Ly) h += 0.5 * (p1 - p0) * (p1 - p0);
                }
                if (x >= 0 && y >= 0) {
                    double p1 = (z + 1 < Lz) ? phi[x + (size_t)Lx * (y + (size_t)Ly * (z + 1))] : 0.0;
                    if (in0 || z + 1 < Lz) h += 0.5 * (p1 - p0) * (p1 - p0);
                }
            }
    return h;
}

/* n_compound compound sweeps, each n_hb heatbath passes then n_or
 * over-relaxation passes.  *pass is the running pass counter (advanced by
 * n_hb + n_or per compound sweep).  If out != NULL, (Q, P, e) is written after
 * every compound sweep: out[3*k + {0,1,2}]. */
void orc_run(double *phi, int Lx, int Ly, int Lz, uint64_t seed, uint32_t chain,
             uint32_t *pass, int n_compound, int n_hb, int n_or,
             const int64_t *site, const double *q, int64_t n, double *out)
{
    for (int k = 0; k < n_compound; ++k) {
        for (int i = 0; i < n_hb; ++i) {
            orc_pass(phi, Lx, Ly, Lz, 1, seed, chain, *pass, 1.0);
            *pass += 1;
        }
        for (int i = 0; i < n_or; ++i) {
            orc_pass(phi, Lx, Ly, Lz, 0, seed, chain, *pass, 1.0);
            *pass += 1;
        }
        if (out) orc_measure(phi, site, q, n, out + 3 * (size_t)k);
    }
}
