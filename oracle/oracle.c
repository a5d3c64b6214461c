/*
 * CPU oracle for the blocked pairwise tensordot -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg call
 * this code.  The GPU library never links, loads or calls it, and it shares
 * no code with the GPU library.
 *
 * Everything is complex128, stored interleaved (re, im) in dense row-major
 * order, and written as plain nested loops so that it can be checked by eye:
 *
 *   oracle_tensordot        the pairwise contraction of Sec. II-A,
 *                           C[fA, fB] = sum_k A[fA, k] B[k, fB], with the
 *                           numpy tensordot conventions (output axes = free
 *                           axes of A in order, then free axes of B in order;
 *                           axes_a[i] is contracted with axes_b[i]).
 *   oracle_block_tensordot  the same contraction computed block by block,
 *                           following the four steps of Sec. II-C: for every
 *                           output block select the A and B blocks by the
 *                           free-index block coordinates, pair them by the
 *                           contracted-index block coordinates, contract each
 *                           pair locally, add the partial into the C block.
 *   oracle_apply_gate1/2    state-vector update by a one- or two-qubit gate
 *                           (Sec. II-A: gates are rank-2 / rank-4 tensors
 *                           acting on the state tensor), used as an
 *                           independent check of network contraction.
 *
 * Return value: 0 on success, -1 on invalid arguments.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXR 128

/* row-major strides (in elements) of a dense tensor */
static void rowmajor_strides(int r, const int64_t *shape, int64_t *st)
{
    int64_t s = 1;
    for (int i = r - 1; i >= 0; --i) {
        st[i] = s;
        s *= shape[i];
    }
}

static int64_t prod(int r, const int64_t *shape)
{
    int64_t p = 1;
    for (int i = 0; i < r; ++i)
        p *= shape[i];
    return p;
}

/* Validate the axes pairing; fill the free-axis lists; return 0 if valid. */
static int classify_axes(int ra, const int64_t *sa, int rb, const int64_t *sb,
                         int naxes, const int *axa, const int *axb,
                         int *fa, int *nfa, int *fb, int *nfb)
{
    int ca[MAXR] = {0}, cb[MAXR] = {0};
    if (ra < 0 || rb < 0 || ra > MAXR || rb > MAXR || naxes < 0 || naxes > ra || naxes > rb)
        return -1;
    for (int i = 0; i < naxes; ++i) {
        if (axa[i] < 0 || axa[i] >= ra || axb[i] < 0 || axb[i] >= rb)
            return -1;
        if (ca[axa[i]] || cb[axb[i]])
            return -1;
        if (sa[axa[i]] != sb[axb[i]])
            return -1;
        ca[axa[i]] = 1;
        cb[axb[i]] = 1;
    }
    *nfa = 0;
    for (int i = 0; i < ra; ++i)
        if (!ca[i])
            fa[(*nfa)++] = i;
    *nfb = 0;
    for (int i = 0; i < rb; ++i)
        if (!cb[i])
            fb[(*nfb)++] = i;
    return 0;
}

/*
 * Plain tensordot.  A, B, C are interleaved complex128 (2 doubles per entry).
 * C has shape (sa[fa[0]], ..., sa[fa[nfa-1]], sb[fb[0]], ..., sb[fb[nfb-1]]).
 * nthreads > 1 splits the output entries over OpenMP threads; the sum over the
 * contracted indices is always taken in the same (row-major) order.
 */
int oracle_tensordot(int ra, const int64_t *sa, const double *A,
                     int rb, const int64_t *sb, const double *B,
                     int naxes, const int *axa, const int *axb,
                     double *C, int nthreads)
{
    int fa[MAXR], fb[MAXR], nfa, nfb;
    int64_t sta[MAXR], stb[MAXR];
    if (classify_axes(ra, sa, rb, sb, naxes, axa, axb, fa, &nfa, fb, &nfb))
        return -1;
    rowmajor_strides(ra, sa, sta);
    rowmajor_strides(rb, sb, stb);

    /* output index space: free axes of A then free axes of B */
    int nout = nfa + nfb;
    int64_t oshape[2 * MAXR], ostride_a[2 * MAXR], ostride_b[2 * MAXR];
    for (int i = 0; i < nfa; ++i) {
        oshape[i] = sa[fa[i]];
        ostride_a[i] = sta[fa[i]];
        ostride_b[i] = 0;
    }
    for (int i = 0; i < nfb; ++i) {
        oshape[nfa + i] = sb[fb[i]];
        ostride_a[nfa + i] = 0;
        ostride_b[nfa + i] = stb[fb[i]];
    }
    /* contracted index space, in the order the axes pairs are given */
    int64_t kshape[MAXR], kstride_a[MAXR], kstride_b[MAXR];
    for (int i = 0; i < naxes; ++i) {
        kshape[i] = sa[axa[i]];
        kstride_a[i] = sta[axa[i]];
        kstride_b[i] = stb[axb[i]];
    }
    int64_t total_out = prod(nout, oshape);
    int64_t total_k = prod(naxes, kshape);

#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t o = 0; o < total_out; ++o) {
        /* decode o (row-major over the output shape) */
        int64_t rem = o, offa = 0, offb = 0;
        for (int i = nout - 1; i >= 0; --i) {
            int64_t d = rem % oshape[i];
            rem /= oshape[i];
            offa += d * ostride_a[i];
            offb += d * ostride_b[i];
        }
        double sre = 0.0, sim = 0.0;
        for (int64_t k = 0; k < total_k; ++k) {
            int64_t kr = k, ka = offa, kb = offb;
            for (int i = naxes - 1; i >= 0; --i) {
                int64_t d = kr % kshape[i];
                kr /= kshape[i];
                ka += d * kstride_a[i];
                kb += d * kstride_b[i];
            }
            double ar = A[2 * ka], ai = A[2 * ka + 1];
            double br = B[2 * kb], bi = B[2 * kb + 1];
            sre += ar * br - ai * bi;
            sim += ar * bi + ai * br;
        }
        C[2 * o] = sre;
        C[2 * o + 1] = sim;
    }
    return 0;
}

/* copy the block with grid coordinate g out of a dense row-major tensor */
static void extract_block(int r, const int64_t *shape, const int64_t *bshape,
                          const int64_t *g, const double *T, double *blk)
{
    int64_t st[MAXR];
    rowmajor_strides(r, shape, st);
    int64_t n = prod(r, bshape);
    for (int64_t e = 0; e < n; ++e) {
        int64_t rem = e, off = 0;
        for (int i = r - 1; i >= 0; --i) {
            int64_t l = rem % bshape[i];
            rem /= bshape[i];
            off += (g[i] * bshape[i] + l) * st[i];
        }
        blk[2 * e] = T[2 * off];
        blk[2 * e + 1] = T[2 * off + 1];
    }
}

/*
 * Blocked tensordot following the steps of Sec. II-C.  Inputs and output are
 * dense row-major (unblocked) tensors; ba, bb are the block shapes (each must
 * divide the shape; contracted axes must have equal block extents).  The
 * output's block shape is the block extents of the free axes.  Computes the
 * same C as oracle_tensordot up to rounding order.
 */
int oracle_block_tensordot(int ra, const int64_t *sa, const int64_t *ba, const double *A,
                           int rb, const int64_t *sb, const int64_t *bb, const double *B,
                           int naxes, const int *axa, const int *axb, double *C)
{
    int fa[MAXR], fb[MAXR], nfa, nfb;
    if (classify_axes(ra, sa, rb, sb, naxes, axa, axb, fa, &nfa, fb, &nfb))
        return -1;
    for (int i = 0; i < ra; ++i)
        if (ba[i] <= 0 || sa[i] % ba[i])
            return -1;
    for (int i = 0; i < rb; ++i)
        if (bb[i] <= 0 || sb[i] % bb[i])
            return -1;
    for (int i = 0; i < naxes; ++i)
        if (ba[axa[i]] != bb[axb[i]])
            return -1;

    int rc = nfa + nfb;
    int64_t sc[2 * MAXR], bc[2 * MAXR], gridc[2 * MAXR], stc[2 * MAXR];
    for (int i = 0; i < nfa; ++i) {
        sc[i] = sa[fa[i]];
        bc[i] = ba[fa[i]];
    }
    for (int i = 0; i < nfb; ++i) {
        sc[nfa + i] = sb[fb[i]];
        bc[nfa + i] = bb[fb[i]];
    }
    for (int i = 0; i < rc; ++i)
        gridc[i] = sc[i] / bc[i];
    rowmajor_strides(rc, sc, stc);

    int64_t gridk[MAXR];
    for (int i = 0; i < naxes; ++i)
        gridk[i] = sa[axa[i]] / ba[axa[i]];
    int64_t nblk_c = prod(rc, gridc), nblk_k = prod(naxes, gridk);
    int64_t na = prod(ra, ba), nb = prod(rb, bb), nc = prod(rc, bc);

    double *blk_a = malloc(sizeof(double) * 2 * (size_t)na);
    double *blk_b = malloc(sizeof(double) * 2 * (size_t)nb);
    double *part = malloc(sizeof(double) * 2 * (size_t)nc);
    double *acc = malloc(sizeof(double) * 2 * (size_t)nc);
    if (!blk_a || !blk_b || !part || !acc) {
        free(blk_a); free(blk_b); free(part); free(acc);
        return -1;
    }

    int64_t gc[2 * MAXR], ga[MAXR], gb[MAXR], gk[MAXR];
    for (int64_t oc = 0; oc < nblk_c; ++oc) {
        /* output block coordinate */
        int64_t rem = oc;
        for (int i = rc - 1; i >= 0; --i) {
            gc[i] = rem % gridc[i];
            rem /= gridc[i];
        }
        /* step 1: the free-index block coordinates select A's and B's blocks */
        for (int i = 0; i < nfa; ++i)
            ga[fa[i]] = gc[i];
        for (int i = 0; i < nfb; ++i)
            gb[fb[i]] = gc[nfa + i];
        memset(acc, 0, sizeof(double) * 2 * (size_t)nc);
        /* step 2: pair them by the contracted-index block coordinates */
        for (int64_t p = 0; p < nblk_k; ++p) {
            int64_t kr = p;
            for (int i = naxes - 1; i >= 0; --i) {
                gk[i] = kr % gridk[i];
                kr /= gridk[i];
            }
            for (int i = 0; i < naxes; ++i) {
                ga[axa[i]] = gk[i];
                gb[axb[i]] = gk[i];
            }
            extract_block(ra, sa, ba, ga, A, blk_a);
            extract_block(rb, sb, bb, gb, B, blk_b);
            /* step 3: local contraction of the coupled pair */
            if (oracle_tensordot(ra, ba, blk_a, rb, bb, blk_b, naxes, axa, axb, part, 1)) {
                free(blk_a); free(blk_b); free(part); free(acc);
                return -1;
            }
            /* step 4: add the partial block into the accumulator */
            for (int64_t e = 0; e < 2 * nc; ++e)
                acc[e] += part[e];
        }
        /* write the finished block into the dense output */
        for (int64_t e = 0; e < nc; ++e) {
            int64_t er = e, off = 0;
            for (int i = rc - 1; i >= 0; --i) {
                int64_t l = er % bc[i];
                er /= bc[i];
                off += (gc[i] * bc[i] + l) * stc[i];
            }
            C[2 * off] = acc[2 * e];
            C[2 * off + 1] = acc[2 * e + 1];
        }
    }
    free(blk_a); free(blk_b); free(part); free(acc);
    return 0;
}

/*
 * State-vector update psi <- G psi for a one-qubit gate G[out,in] (2x2,
 * interleaved complex) on qubit q of an n-qubit state (qubit 0 = most
 * significant bit of the row-major index).
 */
int oracle_apply_gate1(int n, double *psi, int q, const double *G)
{
    if (n < 1 || n > 62 || q < 0 || q >= n)
        return -1;
    int64_t dim = (int64_t)1 << n;
    int64_t bit = (int64_t)1 << (n - 1 - q);
    for (int64_t i = 0; i < dim; ++i) {
        if (i & bit)
            continue;
        int64_t idx[2] = {i, i | bit};
        double in[4] = {psi[2 * idx[0]], psi[2 * idx[0] + 1], psi[2 * idx[1]], psi[2 * idx[1] + 1]};
        for (int o = 0; o < 2; ++o) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < 2; ++j) {
                double gr = G[2 * (2 * o + j)], gi = G[2 * (2 * o + j) + 1];
                re += gr * in[2 * j] - gi * in[2 * j + 1];
                im += gr * in[2 * j + 1] + gi * in[2 * j];
            }
            psi[2 * idx[o]] = re;
            psi[2 * idx[o] + 1] = im;
        }
    }
    return 0;
}

/*
 * State-vector update by a two-qubit gate G[o1,o2,i1,i2] (4x4 matrix with row
 * 2*o1+o2 and column 2*i1+i2, interleaved complex) on qubits (q1, q2).
 */
int oracle_apply_gate2(int n, double *psi, int q1, int q2, const double *G)
{
    if (n < 2 || n > 62 || q1 < 0 || q1 >= n || q2 < 0 || q2 >= n || q1 == q2)
        return -1;
    int64_t dim = (int64_t)1 << n;
    int64_t b1 = (int64_t)1 << (n - 1 - q1);
    int64_t b2 = (int64_t)1 << (n - 1 - q2);
    for (int64_t i = 0; i < dim; ++i) {
        if ((i & b1) || (i & b2))
            continue;
        int64_t idx[4] = {i, i | b2, i | b1, i | b1 | b2}; /* (i1,i2) = 00,01,10,11 */
        double in[8];
        for (int j = 0; j < 4; ++j) {
            in[2 * j] = psi[2 * idx[j]];
            in[2 * j + 1] = psi[2 * idx[j] + 1];
        }
        for (int o = 0; o < 4; ++o) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < 4; ++j) {
                double gr = G[2 * (4 * o + j)], gi = G[2 * (4 * o + j) + 1];
                re += gr * in[2 * j] - gi * in[2 * j + 1];
                im += gr * in[2 * j + 1] + gi * in[2 * j];
            }
            psi[2 * idx[o]] = re;
            psi[2 * idx[o] + 1] = im;
        }
    }
    return 0;
}
