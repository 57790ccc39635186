/*
 * fskmc_oracle.c -- plain CPU restatement of the fractional-step (FS) parallel
 * kinetic Monte Carlo method of Arampatzis, Katsoulakis, Plechac, Taufer and
 * Xu, "Hierarchical fractional-step approximations and parallel kinetic Monte
 * Carlo algorithms" (arXiv:1105.4673).
 *
 * TEST INFRASTRUCTURE. This is the oracle the CUDA library is checked
 * against. Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load it. It shares no code, header, table or helper with
 * the CUDA library, and the library never calls it.
 *
 * It is slow on purpose: before every event the rate-class counts are
 * recounted from scratch, the total rate is re-accumulated, and the chosen
 * member is found by walking the cell in canonical order. All floating point
 * is IEEE binary64; build with -ffp-contract=off so that no multiply-add is
 * fused behind our back (the fma() calls below are the only fused ones).
 *
 * What pins each part (the tests under tests/ do the pinning):
 *   orc_philox       an independent library implementation of Philox4x32-10
 *   orc_rates        the paper's rate formulas (Eq. adsdesrate, Eq. Arrhenius,
 *                    Table COrates) re-derived per site, and detailed balance
 *   orc_fs_run       exact Lie / Strang / random operator products on 4x4
 *                    lattices (chi-square); the J=0 closed form; Onsager
 *   orc_ssa_run      exact e^{TQ} on 3x3 (chi-square); the J=0 closed form
 *   orc_ssa_bkl_run  exact e^{TQ} on 3x3 (chi-square); observables equal to
 *                    orc_ssa_run's over replicas (the class-list form)
 *   orc_observables  brute-force recount in numpy
 *   orc_fs_run_threads  equal, lattice for lattice, to orc_fs_run (the cells
 *                    of one colour are independent, Eq. exact)
 *   orc_fs2_run      exact nested operator products (Eq. opdecomp2) on a 4x4
 *                    lattice (chi-square); the Trotter limit of the inner
 *                    splitting on the exact products
 *
 * Conventions (the paper is silent on all of these; the readings are the
 * project's contract and are shared, by specification only, with the CUDA
 * library):
 *   lattice   periodic lx*ly, site (x,y) has index y*lx+x, one byte per site;
 *             neighbour directions in the order N=(0,-1) E=(+1,0) S=(0,+1)
 *             W=(-1,0).
 *   cells     qx*qy, cell (cx,cy) has id m = cy*ncx+cx; colour E (0) iff
 *             cx+cy is even, O (1) otherwise (the checkerboard, Eq. sublatt).
 *   events    a site event belongs to the cell holding the site (Eq.
 *             gendecomp). A bond inside a cell belongs to that cell. A bond
 *             crossing a vertical cell edge (horizontal bond) belongs to the
 *             E cell and runs in E windows; a bond crossing a horizontal cell
 *             edge (vertical bond) belongs to the O cell and runs in O windows.
 *   members   site members in local row-major order; bond members are
 *             directed slots (s,d) taken s-major then d: d=0..3 is the
 *             outward event s->s+dir(d), d=4..7 the inward event
 *             s+dir(d-4)->s from a halo origin; a slot exists only if the
 *             cell owns it.
 *   RNG       Philox4x32-10, key (seed lo, seed hi), counter
 *             (e, w, m, replica | tag<<24); tags 0 event, 1 serial SSA,
 *             2 initial state, 3 schedule.
 *   draws     u_t = ((w0<<21 | w1>>11) + 1) * 2^-53 in (0,1];
 *             u_c = (w2 + 0.5) * 2^-32; member j = (w3 * n_k) >> 32.
 *   windows   a cell reads outside its write set from the lattice as it was
 *             when the window began, and reads and writes its write set
 *             through a private copy; the pending event that would cross the
 *             window edge is discarded.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ADSDES 0
#define ORC_ISING 1
#define ORC_DIFFUSION 2
#define ORC_ZGB 3
#define ORC_ISING1D 4

#define ORC_LIE 0
#define ORC_STRANG 1
#define ORC_RANDOM 2
#define ORC_RANDOM_ORDER 3

#define TAG_EVENT 0u
#define TAG_SSA 1u
#define TAG_INIT 2u
#define TAG_SCHED 3u

#define ORC_EDGE_TOL 1e-12

static const int DX[4] = {0, 1, 0, -1};
static const int DY[4] = {-1, 0, 1, 0};

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies, the    */
/* high halves xored into the other two words with the round key; the key   */
/* advances by the Weyl constants between rounds.                           */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                 uint32_t out[4])
{
    uint32_t ctr[4] = {a, b, c, d};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Models and rates.                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int lx, ly, qx, qy, ncx, ncy;
    int model, nclass, slots;
    double r[16];
} sys_t;

/*
 * Rate of each class, in class order.
 *  ADSDES  (adsorption/desorption spin flip, Eq. adsdesrate with J(x-y)=J on
 *          nearest neighbours): class 5*sigma+n, n = occupied neighbours;
 *          r(0,n) = ka, r(1,n) = kd*exp(-betaJ*n).
 *  ISING   (spin-flip Arrhenius dynamics, Eq. Arrhenius, with U = K*n - h,
 *          K = 4J and the zero-field value h = 2K of Section 7): same 10
 *          classes; r(0,n) = ka, r(1,n) = kd*exp(-4*betaJ*(n-2)).
 *  DIFFUSION (adsorption/desorption plus nearest-neighbour hops, Section 2
 *          example 2): classes 0-9 as ADSDES; 10+n is a directed slot whose
 *          origin is occupied with n occupied neighbours and whose target is
 *          empty, rate nu*exp(-betaJ*n).
 *  ISING1D (the 1D Ising benchmark of Section 7 on a ring, ly = 1, with
 *          H = -K sum sigma(x) sigma(x+1) + h sum sigma(x), betaJ = beta K,
 *          betah = beta h; detailed balance as for ISING): class 3*sigma + n,
 *          n = occupied east/west neighbours; r(0,n) = ka,
 *          r(1,n) = kd*exp(-(beta K n - beta h)).
 *  ZGB     (Table COrates; states 0 empty, 1 A, 2 B): 0 A adsorbs on an empty
 *          site (yA); 1 B2 adsorbs on a directed slot with both ends empty
 *          ((1-yA)/4); 2 A+B react on a directed slot holding (A,B) or (B,A)
 *          (kr/4); 3 A desorbs (kd).
 * Returns the number of classes, or -1 for an unknown model.
 */
int orc_rates(int model, double ka, double kd, double betaJ, double nu,
              double yA, double kr, double betah, double *r)
{
    int n;
    switch (model) {
    case ORC_ISING1D:
        for (n = 0; n < 3; n++) {
            r[n] = ka;
            r[3 + n] = kd * exp(-(betaJ * (double)n - betah));
        }
        return 6;
    case ORC_ADSDES:
        for (n = 0; n < 5; n++) {
            r[n] = ka;
            r[5 + n] = kd * exp(-(betaJ * (double)n));
        }
        return 10;
    case ORC_ISING:
        for (n = 0; n < 5; n++) {
            r[n] = ka;
            r[5 + n] = kd * exp(-(4.0 * betaJ) * (double)(n - 2));
        }
        return 10;
    case ORC_DIFFUSION:
        for (n = 0; n < 5; n++) {
            r[n] = ka;
            r[5 + n] = kd * exp(-(betaJ * (double)n));
            r[10 + n] = nu * exp(-(betaJ * (double)n));
        }
        return 15;
    case ORC_ZGB:
        r[0] = yA;
        r[1] = (1.0 - yA) * 0.25;
        r[2] = kr * 0.25;
        r[3] = kd;
        return 4;
    }
    return -1;
}

static int sys_init(sys_t *S, int lx, int ly, int qx, int qy, int model,
                    const double *rates7)
{
    memset(S, 0, sizeof(*S));
    S->lx = lx; S->ly = ly; S->qx = qx; S->qy = qy;
    S->ncx = qx > 0 ? lx / qx : 0;
    S->ncy = qy > 0 ? ly / qy : 0;
    S->model = model;
    S->nclass = orc_rates(model, rates7[0], rates7[1], rates7[2], rates7[3],
                          rates7[4], rates7[5], rates7[6], S->r);
    S->slots = (model == ORC_DIFFUSION || model == ORC_ZGB);
    return S->nclass > 0 ? 0 : -1;
}

/* Cell geometry: lx % 2qx == 0 and ly % 2qy == 0 (a checkerboard of
 * cells); the 1D ring has ly == qy == 1 (cells alternate along x). */
static int geometry_ok(int model, int lx, int ly, int qx, int qy)
{
    if (qx < 1 || qy < 1 || lx % (2 * qx)) return 0;
    if (model == ORC_ISING1D) return ly == 1 && qy == 1;
    return ly % (2 * qy) == 0;
}

static int wrap(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

static int sidx(const sys_t *S, int x, int y)
{
    return wrap(y, S->ly) * S->lx + wrap(x, S->lx);
}

/* ------------------------------------------------------------------------ */
/* A view of the lattice during one cell's window: the write set is read    */
/* and written through `priv`, everything else is read from `snap`.         */
/* Membership in the write set is marked by stamp[i] == cur.                */
/* ------------------------------------------------------------------------ */
typedef struct {
    const sys_t *S;
    const uint8_t *snap;
    uint8_t *priv;
    uint32_t *stamp;
    uint32_t cur;
} view_t;

static int vget(const view_t *v, int i)
{
    return v->stamp[i] == v->cur ? v->priv[i] : v->snap[i];
}

static void vset(view_t *v, int i, int val)
{
    v->priv[i] = (uint8_t)val;
}

/* number of nearest neighbours of site (x,y) in state 1 */
static int occ_nbrs(const view_t *v, int x, int y)
{
    int n = 0;
    for (int d = 0; d < 4; d++)
        n += vget(v, sidx(v->S, x + DX[d], y + DY[d])) == 1;
    return n;
}

static int site_class(const view_t *v, int x, int y)
{
    int s = vget(v, sidx(v->S, x, y));
    switch (v->S->model) {
    case ORC_ISING1D:
        return 3 * s + (vget(v, sidx(v->S, x - 1, y)) == 1) + (vget(v, sidx(v->S, x + 1, y)) == 1);
    case ORC_ADSDES:
    case ORC_ISING:
    case ORC_DIFFUSION:
        return 5 * s + occ_nbrs(v, x, y);
    case ORC_ZGB:
        return s == 0 ? 0 : (s == 1 ? 3 : -1);
    }
    return -1;
}

static int slot_class(const view_t *v, int ox, int oy, int tx, int ty)
{
    int so = vget(v, sidx(v->S, ox, oy));
    int st = vget(v, sidx(v->S, tx, ty));
    switch (v->S->model) {
    case ORC_DIFFUSION:
        return (so == 1 && st == 0) ? 10 + occ_nbrs(v, ox, oy) : -1;
    case ORC_ZGB:
        if (so == 0 && st == 0) return 1;
        if ((so == 1 && st == 2) || (so == 2 && st == 1)) return 2;
        return -1;
    }
    return -1;
}

/* A member: a site (kind 0) or a directed slot origin->target (kind 1),
 * in global coordinates (unwrapped; wrap on access). */
typedef struct {
    int kind, ox, oy, tx, ty, cls;
} member_t;

static int horizontal(int dir) { return dir == 1 || dir == 3; }

/*
 * List the members a cell owns in a window of colour `col`, in canonical
 * order, with their current classes (the owned part of Eq. gendecomp for
 * cell m, restricted to the cell's colour as in Eq. opdecomp). A bond that
 * crosses a cell edge is owned only in the window named by the ownership
 * rule in the header. Returns the number written (<= 9*qx*qy).
 */
static int cell_members(const view_t *v, int cx, int cy, int col, member_t *out)
{
    const sys_t *S = v->S;
    int cnt = 0, X0 = cx * S->qx, Y0 = cy * S->qy;
    for (int ly = 0; ly < S->qy; ly++)
        for (int lx = 0; lx < S->qx; lx++) {
            int x = X0 + lx, y = Y0 + ly;
            member_t *mb = &out[cnt++];
            mb->kind = 0; mb->ox = x; mb->oy = y; mb->tx = x; mb->ty = y;
            mb->cls = site_class(v, x, y);
            if (!S->slots) continue;
            for (int d = 0; d < 8; d++) {
                int dir = d & 3, inward = d >= 4;
                int nlx = lx + DX[dir], nly = ly + DY[dir];
                int inside = nlx >= 0 && nlx < S->qx && nly >= 0 && nly < S->qy;
                int cross_owned = horizontal(dir) ? (col == 0) : (col == 1);
                int owned = inward ? (!inside && cross_owned) : (inside || cross_owned);
                if (!owned) continue;
                member_t *b = &out[cnt++];
                b->kind = 1;
                if (!inward) { b->ox = x; b->oy = y; b->tx = x + DX[dir]; b->ty = y + DY[dir]; }
                else { b->ox = x + DX[dir]; b->oy = y + DY[dir]; b->tx = x; b->ty = y; }
                b->cls = slot_class(v, b->ox, b->oy, b->tx, b->ty);
            }
        }
    return cnt;
}

/* Write set of a cell in a window of colour col: its own sites and, for
 * models with bond events, the halo ends of the cross bonds it owns.
 * Returns count; out holds site indices. */
static int cell_writeset(const sys_t *S, int cx, int cy, int col, int *out)
{
    int cnt = 0, X0 = cx * S->qx, Y0 = cy * S->qy;
    for (int ly = 0; ly < S->qy; ly++)
        for (int lx = 0; lx < S->qx; lx++)
            out[cnt++] = sidx(S, X0 + lx, Y0 + ly);
    if (!S->slots) return cnt;
    if (col == 0) {
        for (int ly = 0; ly < S->qy; ly++) {
            out[cnt++] = sidx(S, X0 - 1, Y0 + ly);
            out[cnt++] = sidx(S, X0 + S->qx, Y0 + ly);
        }
    } else {
        for (int lx = 0; lx < S->qx; lx++) {
            out[cnt++] = sidx(S, X0 + lx, Y0 - 1);
            out[cnt++] = sidx(S, X0 + lx, Y0 + S->qy);
        }
    }
    return cnt;
}

/* Apply the event of a member of class k (the update sigma -> sigma^{x,omega}
 * of Section 2's examples). */
static void apply_member(view_t *v, const member_t *mb, int k)
{
    const sys_t *S = v->S;
    int io = sidx(S, mb->ox, mb->oy), it = sidx(S, mb->tx, mb->ty);
    switch (S->model) {
    case ORC_ADSDES:
    case ORC_ISING:
    case ORC_ISING1D:
        vset(v, io, 1 - vget(v, io));
        break;
    case ORC_DIFFUSION:
        if (k < 10) vset(v, io, 1 - vget(v, io));
        else { vset(v, io, 0); vset(v, it, 1); }
        break;
    case ORC_ZGB:
        if (k == 0) vset(v, io, 1);
        else if (k == 1) { vset(v, io, 2); vset(v, it, 2); }
        else if (k == 2) { vset(v, io, 0); vset(v, it, 0); }
        else vset(v, io, 0);
        break;
    }
}

/* ------------------------------------------------------------------------ */
/* The SSA kernel: Eq. totalrate (total rate), an exponential waiting time, */
/* and Eq. skeleton (event chosen with probability c/lambda). `members`     */
/* lists the candidate events; classes are recounted on every call.         */
/* Returns: 0 event applied, 1 window over, 2 no event possible.            */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t seed;
    uint32_t c1, c2, c3; /* counter words after the event index */
} stream_t;

static int ssa_step(view_t *v, member_t *mb, int nmb, double *tau, double h,
                    uint32_t e, const stream_t *st, int *ambiguous)
{
    const sys_t *S = v->S;
    int64_t n[16] = {0};
    for (int i = 0; i < nmb; i++)
        if (mb[i].cls >= 0) n[mb[i].cls]++;

    double lam = 0.0;
    for (int k = 0; k < S->nclass; k++)
        lam = fma((double)n[k], S->r[k], lam);
    if (lam == 0.0) return 2;

    uint32_t o[4];
    draw(st->seed, e, st->c1, st->c2, st->c3, o);
    uint64_t b53 = ((uint64_t)o[0] << 21) | (uint64_t)(o[1] >> 11);
    double ut = (double)(b53 + 1) * 0x1p-53;
    double E = -log(ut) / lam;
    double end = *tau + E;
    if (fabs(end - h) < ORC_EDGE_TOL * h) *ambiguous = 1;
    if (end >= h) return 1;
    *tau = end;

    double uc = ((double)o[2] + 0.5) * 0x1p-32;
    double t = uc * lam;
    double P = 0.0;
    int k;
    for (k = 0; k < S->nclass; k++) {
        P = fma((double)n[k], S->r[k], P);
        if (t < P) break;
    }
    uint32_t j = (uint32_t)(((uint64_t)o[3] * (uint64_t)n[k]) >> 32);
    for (int i = 0; i < nmb; i++)
        if (mb[i].cls == k) {
            if (j == 0) { apply_member(v, &mb[i], k); return 0; }
            j--;
        }
    return 2; /* unreachable: n[k] > 0 members of class k exist */
}

/* ------------------------------------------------------------------------ */
/* The fractional-step window for one cell (Step 1 / Step 3 of Section 2.2: */
/* a serial KMC kernel on the cell for the window length h).                */
/* ------------------------------------------------------------------------ */
typedef struct {
    sys_t S;
    uint8_t *snap, *priv;
    uint32_t *stamp;
    uint32_t cur;
    member_t *mb;
    int *ws;
} work_t;

static int work_init(work_t *W, const sys_t *S)
{
    size_t N = (size_t)S->lx * S->ly;
    W->S = *S;
    W->snap = (uint8_t *)malloc(N);
    W->priv = (uint8_t *)malloc(N);
    W->stamp = (uint32_t *)calloc(N, sizeof(uint32_t));
    W->cur = 0;
    W->mb = (member_t *)malloc(sizeof(member_t) * (size_t)(9 * S->qx * S->qy + 8));
    W->ws = (int *)malloc(sizeof(int) * (size_t)(S->qx * S->qy + 2 * (S->qx + S->qy) + 8));
    return (W->snap && W->priv && W->stamp && W->mb && W->ws) ? 0 : -1;
}

static void work_free(work_t *W)
{
    free(W->snap); free(W->priv); free(W->stamp); free(W->mb); free(W->ws);
}

/* Run one cell's window against W->snap, write its write set into lat. */
static uint32_t cell_window(work_t *W, uint8_t *lat, int cx, int cy, int col,
                            double h, uint32_t w, uint32_t rep, uint64_t seed,
                            int *ambiguous)
{
    const sys_t *S = &W->S;
    uint32_t m = (uint32_t)(cy * S->ncx + cx);
    int nws = cell_writeset(S, cx, cy, col, W->ws);
    W->cur++;
    if (W->cur == 0) { /* stamp counter wrapped: clear and restart */
        memset(W->stamp, 0, sizeof(uint32_t) * (size_t)S->lx * S->ly);
        W->cur = 1;
    }
    for (int i = 0; i < nws; i++) {
        W->stamp[W->ws[i]] = W->cur;
        W->priv[W->ws[i]] = W->snap[W->ws[i]];
    }
    view_t v = {S, W->snap, W->priv, W->stamp, W->cur};
    stream_t st = {seed, w, m, rep | (TAG_EVENT << 24)};
    double tau = 0.0;
    uint32_t e = 0;
    *ambiguous = 0;
    for (;;) {
        int nmb = cell_members(&v, cx, cy, col, W->mb);
        if (ssa_step(&v, W->mb, nmb, &tau, h, e, &st, ambiguous) != 0) break;
        e++;
    }
    for (int i = 0; i < nws; i++)
        lat[W->ws[i]] = W->priv[W->ws[i]];
    return e;
}

/* One fractional window: every cell of colour col advances by h, reading
 * the lattice as it was when the window began (Eq. exact: the same-colour
 * cell generators commute, so the cell order does not matter; `order`
 * selects forward (0) or reverse (1) to let tests check that). */
static void window_all(work_t *W, uint8_t *lat, int col, double h, uint32_t w,
                       uint32_t rep, uint64_t seed, int order, uint64_t *events,
                       uint64_t *amb, int32_t *workload)
{
    const sys_t *S = &W->S;
    size_t N = (size_t)S->lx * S->ly;
    int nc = S->ncx * S->ncy;
    memcpy(W->snap, lat, N);
    for (int ii = 0; ii < nc; ii++) {
        int m = order ? nc - 1 - ii : ii;
        int cx = m % S->ncx, cy = m / S->ncx;
        if (((cx + cy) & 1) != col) continue;
        int a = 0;
        uint32_t e = cell_window(W, lat, cx, cy, col, h, w, rep, seed, &a);
        *events += e;
        *amb += (uint64_t)a;
        if (workload) workload[m] = (int32_t)e;
    }
}

/* ------------------------------------------------------------------------ */
/* Processor communication schedules (Section 3).                           */
/*  LIE          E(dt) O(dt) per step (Eq. lie, E first as in Steps 1-3)    */
/*  STRANG       E(dt/2) O(dt) E(dt/2) per step (Eq. strang)                */
/*  RANDOM       2T/dt windows of length dt, colour drawn fair per window   */
/*               (Eq. SLPCS; the averaged generator is L/2, so two windows  */
/*               of length dt advance the physical clock by dt)             */
/*  RANDOM_ORDER per step, (E,O) or (O,E) with probability 1/2, each dt     */
/* The colour bit for a window or step starting at global window index w is */
/* bit 0 of word 0 of Philox(seed, (0, w, 0, replica | 3<<24)); 0 means E.  */
/* Returns the number of windows, or -1 if T/dt is not an integer.          */
/* ------------------------------------------------------------------------ */
static int64_t nsteps(double dt, double T)
{
    if (!(dt > 0.0) || !(T >= 0.0)) return -1;
    double q = T / dt;
    double n = floor(q + 0.5);
    if (fabs(n * dt - T) > 1e-9 * T) return -1;
    return (int64_t)n;
}

int64_t orc_schedule(int scheme, double dt, double T, uint64_t seed, uint32_t rep,
                     uint32_t w0, int32_t *colour, double *h, int64_t cap)
{
    int64_t n = nsteps(dt, T), cnt = 0;
    if (n < 0 || scheme < 0 || scheme > 3) return -1;
    int64_t total = scheme == ORC_STRANG ? 3 * n : 2 * n;
    if (colour == NULL) return total;
    if (total > cap) return -1;
    for (int64_t i = 0; i < n; i++) {
        uint32_t o[4];
        uint32_t w = w0 + (uint32_t)cnt;
        switch (scheme) {
        case ORC_LIE:
            colour[cnt] = 0; h[cnt++] = dt;
            colour[cnt] = 1; h[cnt++] = dt;
            break;
        case ORC_STRANG:
            colour[cnt] = 0; h[cnt++] = dt * 0.5;
            colour[cnt] = 1; h[cnt++] = dt;
            colour[cnt] = 0; h[cnt++] = dt * 0.5;
            break;
        case ORC_RANDOM:
            draw(seed, 0, w, 0, rep | (TAG_SCHED << 24), o);
            colour[cnt] = (int32_t)(o[0] & 1u); h[cnt++] = dt;
            draw(seed, 0, w + 1, 0, rep | (TAG_SCHED << 24), o);
            colour[cnt] = (int32_t)(o[0] & 1u); h[cnt++] = dt;
            break;
        case ORC_RANDOM_ORDER:
            draw(seed, 0, w, 0, rep | (TAG_SCHED << 24), o);
            colour[cnt] = (int32_t)(o[0] & 1u); h[cnt++] = dt;
            colour[cnt] = (int32_t)(1u - (o[0] & 1u)); h[cnt++] = dt;
            break;
        }
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points (argument meaning is in oracle/__init__.py).       */
/* rates7 = {ka, kd, betaJ, nu, yA, kr}.                                    */
/* ------------------------------------------------------------------------ */

/* Bernoulli(p) initial state: site i of replica rep is 1 iff word 0 of
 * Philox(seed, (i, 0, 0, rep | 2<<24)) < p * 2^32. */
void orc_init_bernoulli(int lx, int ly, uint64_t seed, double p, uint32_t rep,
                        uint8_t *lat)
{
    double thr = p * 4294967296.0;
    for (int64_t i = 0; i < (int64_t)lx * ly; i++) {
        uint32_t o[4];
        draw(seed, (uint32_t)i, 0, 0, rep | (TAG_INIT << 24), o);
        lat[i] = (double)o[0] < thr ? 1 : 0;
    }
}

/* Gaussian-bump pre-coverage: site (x,y) holds species `species` with
 * probability amp * g(dx) * g(dy), g(d) = exp(-d*d / (2*s*s)), s = width,
 * d the periodic distance to the centre (x0,y0) = (word0 mod lx, word1 mod
 * ly) of Philox(seed, (0, 0xFFFFFFFF, 0, rep | 3<<24)); empty otherwise.
 * The draw per site is the Bernoulli draw above. */
void orc_init_bump(int lx, int ly, uint64_t seed, double amp, double width,
                   int species, uint32_t rep, uint8_t *lat)
{
    uint32_t c[4];
    draw(seed, 0, 0xFFFFFFFFu, 0, rep | (TAG_SCHED << 24), c);
    int x0 = (int)(c[0] % (uint32_t)lx), y0 = (int)(c[1] % (uint32_t)ly);
    double *gx = (double *)malloc(sizeof(double) * (size_t)lx);
    double *gy = (double *)malloc(sizeof(double) * (size_t)ly);
    double two_s2 = 2.0 * width * width;
    for (int x = 0; x < lx; x++) {
        int d = abs(x - x0);
        if (lx - d < d) d = lx - d;
        gx[x] = exp(-((double)d * (double)d) / two_s2);
    }
    for (int y = 0; y < ly; y++) {
        int d = abs(y - y0);
        if (ly - d < d) d = ly - d;
        gy[y] = exp(-((double)d * (double)d) / two_s2);
    }
    for (int y = 0; y < ly; y++)
        for (int x = 0; x < lx; x++) {
            int64_t i = (int64_t)y * lx + x;
            uint32_t o[4];
            draw(seed, (uint32_t)i, 0, 0, rep | (TAG_INIT << 24), o);
            double p = (amp * gx[x]) * gy[y];
            lat[i] = (double)o[0] < p * 4294967296.0 ? (uint8_t)species : 0;
        }
    free(gx);
    free(gy);
}

/*
 * Run the FS scheme for time T from global window index *w (updated on
 * return), in place on lat. stats_out = {events, windows, ambiguous};
 * workload (ncx*ncy, may be NULL) receives each cell's event count in its
 * latest window. Returns 0, or -1 on invalid arguments.
 */
int orc_fs_run(int lx, int ly, int qx, int qy, int model, const double *rates7,
               int scheme, double dt, double T, uint64_t seed, uint32_t rep,
               uint32_t *w, int order, uint8_t *lat, uint64_t *stats_out,
               int32_t *workload)
{
    sys_t S;
    if (!geometry_ok(model, lx, ly, qx, qy)) return -1;
    if (sys_init(&S, lx, ly, qx, qy, model, rates7)) return -1;
    int64_t nw = orc_schedule(scheme, dt, T, seed, rep, *w, NULL, NULL, 0);
    if (nw < 0) return -1;
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nw + 1));
    double *hh = (double *)malloc(sizeof(double) * (size_t)(nw + 1));
    orc_schedule(scheme, dt, T, seed, rep, *w, col, hh, nw);
    work_t W;
    if (work_init(&W, &S)) { work_free(&W); free(col); free(hh); return -1; }
    uint64_t ev = 0, amb = 0;
    for (int64_t i = 0; i < nw; i++)
        window_all(&W, lat, col[i], hh[i], *w + (uint32_t)i, rep, seed, order,
                   &ev, &amb, workload);
    *w += (uint32_t)nw;
    stats_out[0] += ev;
    stats_out[1] += (uint64_t)nw;
    stats_out[2] += amb;
    work_free(&W);
    free(col);
    free(hh);
    return 0;
}

/* One window of colour col and length h at global index w (for per-window
 * comparisons). amb_cells (ncx*ncy, may be NULL) gets 1 for cells whose
 * window was flagged ambiguous. */
int orc_window(int lx, int ly, int qx, int qy, int model, const double *rates7,
               int col, double h, uint32_t w, uint64_t seed, uint32_t rep,
               uint8_t *lat, uint64_t *stats_out, int32_t *workload,
               int32_t *amb_cells)
{
    sys_t S;
    if (!geometry_ok(model, lx, ly, qx, qy)) return -1;
    if (sys_init(&S, lx, ly, qx, qy, model, rates7)) return -1;
    work_t W;
    if (work_init(&W, &S)) { work_free(&W); return -1; }
    size_t N = (size_t)lx * ly;
    memcpy(W.snap, lat, N);
    uint64_t ev = 0, amb = 0;
    for (int m = 0; m < S.ncx * S.ncy; m++) {
        int cx = m % S.ncx, cy = m / S.ncx;
        if (((cx + cy) & 1) != col) continue;
        int a = 0;
        uint32_t e = cell_window(&W, lat, cx, cy, col, h, w, rep, seed, &a);
        ev += e;
        amb += (uint64_t)a;
        if (workload) workload[m] = (int32_t)e;
        if (amb_cells) amb_cells[m] = a;
    }
    stats_out[0] += ev;
    stats_out[1] += 1;
    stats_out[2] += amb;
    work_free(&W);
    return 0;
}

/*
 * Serial Gillespie SSA over the whole lattice for time T (the process the
 * FS scheme approximates, Eq. generator, simulated by Eqs. totalrate and
 * skeleton). Every site and every directed nearest-neighbour bond is a
 * candidate; classes and rates are the FS classes. Draws use counter
 * (e lo, e hi, 0, rep | 1<<24). The total rate is recounted every event
 * (the direct method, O(N) per event). Returns the number of events.
 */
int64_t orc_ssa_run(int lx, int ly, int model, const double *rates7, double T,
                    uint64_t seed, uint32_t rep, uint8_t *lat)
{
    sys_t S;
    if (sys_init(&S, lx, ly, lx, ly, model, rates7)) return -1;
    size_t N = (size_t)lx * ly;
    member_t *mb = (member_t *)malloc(sizeof(member_t) * (N * 5 + 1));
    uint32_t *stamp = (uint32_t *)calloc(N, sizeof(uint32_t));
    if (!mb || !stamp) { free(mb); free(stamp); return -1; }
    for (size_t i = 0; i < N; i++) stamp[i] = 1; /* the whole lattice is writable */
    view_t v = {&S, lat, lat, stamp, 1};
    double tau = 0.0;
    uint64_t e = 0;
    int amb = 0;
    for (;;) {
        int nmb = 0;
        for (int y = 0; y < ly; y++)
            for (int x = 0; x < lx; x++) {
                member_t *a = &mb[nmb++];
                a->kind = 0; a->ox = x; a->oy = y; a->tx = x; a->ty = y;
                a->cls = site_class(&v, x, y);
                if (!S.slots) continue;
                for (int d = 0; d < 4; d++) {
                    member_t *b = &mb[nmb++];
                    b->kind = 1; b->ox = x; b->oy = y;
                    b->tx = x + DX[d]; b->ty = y + DY[d];
                    b->cls = slot_class(&v, x, y, b->tx, b->ty);
                }
            }
        stream_t st = {seed, (uint32_t)(e >> 32), 0, rep | (TAG_SSA << 24)};
        if (ssa_step(&v, mb, nmb, &tau, T, (uint32_t)e, &st, &amb) != 0) break;
        e++;
    }
    free(mb);
    free(stamp);
    return (int64_t)e;
}

/* ------------------------------------------------------------------------ */
/* Serial SSA with class lists (the BKL form, Section 1's reference to      */
/* Bortz-Kalos-Lebowitz): the same classes, rates, draws and time steps as  */
/* orc_ssa_run, but each class keeps an array of its members, updated by    */
/* swap-remove when an event changes a member's class, so an event costs    */
/* O(1) instead of a recount of the lattice. The j-th member of class k is  */
/* the j-th entry of the class's array (an order of its own), so the        */
/* trajectory differs from the direct form's while the law is the same;    */
/* tests cross-check the two (and both against e^{TQ}). Member ids: site i  */
/* is i, the directed slot from site i in direction d is N + 4i + d.        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t *list;  /* nclass lists of capacity M each */
    int32_t *cnt;   /* members per class */
    int32_t *cls;   /* class of each member (-1: none) */
    int32_t *pos;   /* position of each member in its class's list */
    int M;
} bkl_t;

static void bkl_set(bkl_t *B, int m, int k)
{
    int k0 = B->cls[m];
    if (k0 == k) return;
    if (k0 >= 0) { /* swap-remove from the old list */
        int p = B->pos[m], last = B->list[(size_t)k0 * B->M + B->cnt[k0] - 1];
        B->list[(size_t)k0 * B->M + p] = last;
        B->pos[last] = p;
        B->cnt[k0]--;
    }
    if (k >= 0) {
        B->list[(size_t)k * B->M + B->cnt[k]] = m;
        B->pos[m] = B->cnt[k]++;
    }
    B->cls[m] = k;
}

/* the class of member m on the whole lattice */
static int bkl_class(const view_t *v, int m)
{
    const sys_t *S = v->S;
    int N = S->lx * S->ly;
    if (m < N) return site_class(v, m % S->lx, m / S->lx);
    int i = (m - N) >> 2, d = (m - N) & 3;
    int x = i % S->lx, y = i / S->lx;
    return slot_class(v, x, y, x + DX[d], y + DY[d]);
}

/* re-class every member whose class can depend on site c: the sites within
 * one step of c and the slots leaving them (a class depends on the states
 * of its site or slot ends and, for the n-dependent rates, on the states of
 * the origin's neighbours) */
static void bkl_touch(bkl_t *B, const view_t *v, int c)
{
    const sys_t *S = v->S;
    int N = S->lx * S->ly, cx = c % S->lx, cy = c / S->lx;
    for (int k = -1; k < 4; k++) {
        int x = k < 0 ? cx : cx + DX[k], y = k < 0 ? cy : cy + DY[k];
        if (S->model == ORC_ISING1D && y != cy) continue;
        int i = sidx(S, x, y);
        bkl_set(B, i, bkl_class(v, i));
        if (S->slots)
            for (int d = 0; d < 4; d++) bkl_set(B, N + 4 * i + d, bkl_class(v, N + 4 * i + d));
    }
}

int64_t orc_ssa_bkl_run(int lx, int ly, int model, const double *rates7, double T,
                        uint64_t seed, uint32_t rep, uint8_t *lat)
{
    sys_t S;
    if (sys_init(&S, lx, ly, lx, ly, model, rates7)) return -1;
    int N = lx * ly, M = S.slots ? 5 * N : N;
    bkl_t B;
    B.M = M;
    B.list = (int32_t *)malloc(sizeof(int32_t) * (size_t)M * (size_t)S.nclass);
    B.cnt = (int32_t *)calloc(16, sizeof(int32_t));
    B.cls = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    B.pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    uint32_t *stamp = (uint32_t *)calloc((size_t)N, sizeof(uint32_t));
    if (!B.list || !B.cnt || !B.cls || !B.pos || !stamp) {
        free(B.list); free(B.cnt); free(B.cls); free(B.pos); free(stamp);
        return -1;
    }
    for (int i = 0; i < N; i++) stamp[i] = 1; /* the whole lattice is writable */
    view_t v = {&S, lat, lat, stamp, 1};
    for (int m = 0; m < M; m++) B.cls[m] = -1;
    for (int m = 0; m < M; m++) {
        if (model == ORC_ISING1D && m >= N) break;
        bkl_set(&B, m, bkl_class(&v, m));
    }
    double tau = 0.0;
    uint64_t e = 0;
    for (;;) {
        double lam = 0.0;
        for (int k = 0; k < S.nclass; k++) lam = fma((double)B.cnt[k], S.r[k], lam);
        if (lam == 0.0) break;
        uint32_t o[4];
        draw(seed, (uint32_t)e, (uint32_t)(e >> 32), 0, rep | (TAG_SSA << 24), o);
        uint64_t b53 = ((uint64_t)o[0] << 21) | (uint64_t)(o[1] >> 11);
        double ut = (double)(b53 + 1) * 0x1p-53;
        double end = tau + (-log(ut) / lam);
        if (end >= T) break;
        tau = end;
        double t = (((double)o[2] + 0.5) * 0x1p-32) * lam;
        double P = 0.0;
        int k;
        for (k = 0; k < S.nclass; k++) {
            P = fma((double)B.cnt[k], S.r[k], P);
            if (t < P) break;
        }
        uint32_t j = (uint32_t)(((uint64_t)o[3] * (uint64_t)B.cnt[k]) >> 32);
        int m = B.list[(size_t)k * M + j];
        member_t mb;
        if (m < N) {
            mb.kind = 0; mb.ox = mb.tx = m % lx; mb.oy = mb.ty = m / lx;
        } else {
            int i = (m - N) >> 2, d = (m - N) & 3;
            mb.kind = 1; mb.ox = i % lx; mb.oy = i / lx; mb.tx = mb.ox + DX[d]; mb.ty = mb.oy + DY[d];
        }
        mb.cls = k;
        apply_member(&v, &mb, k);
        bkl_touch(&B, &v, sidx(&S, mb.ox, mb.oy));
        if (mb.kind == 1) bkl_touch(&B, &v, sidx(&S, mb.tx, mb.ty));
        e++;
    }
    free(B.list); free(B.cnt); free(B.cls); free(B.pos); free(stamp);
    return (int64_t)e;
}

/* Total rate lambda(sigma) of Eq. totalrate over the whole lattice, and the
 * per-class counts (whole-lattice candidate set as in orc_ssa_run). */
double orc_total_rate(int lx, int ly, int model, const double *rates7,
                      const uint8_t *lat, int64_t *counts)
{
    sys_t S;
    if (sys_init(&S, lx, ly, lx, ly, model, rates7)) return -1.0;
    size_t N = (size_t)lx * ly;
    uint32_t *stamp = (uint32_t *)calloc(N, sizeof(uint32_t));
    view_t v = {&S, lat, (uint8_t *)lat, stamp, 1};
    for (int k = 0; k < 16; k++) counts[k] = 0;
    for (int y = 0; y < ly; y++)
        for (int x = 0; x < lx; x++) {
            int c = site_class(&v, x, y);
            if (c >= 0) counts[c]++;
            if (!S.slots) continue;
            for (int d = 0; d < 4; d++) {
                c = slot_class(&v, x, y, x + DX[d], y + DY[d]);
                if (c >= 0) counts[c]++;
            }
        }
    double lam = 0.0;
    for (int k = 0; k < S.nclass; k++) lam = fma((double)counts[k], S.r[k], lam);
    free(stamp);
    return lam;
}

/* Members a cell owns in a window of colour col (for the partition tests):
 * origin and target site indices and class of each, canonical order. */
int orc_cell_members(int lx, int ly, int qx, int qy, int model,
                     const double *rates7, const uint8_t *lat, int m, int col,
                     int32_t *origin, int32_t *target, int32_t *kind,
                     int32_t *cls)
{
    sys_t S;
    if (sys_init(&S, lx, ly, qx, qy, model, rates7)) return -1;
    size_t N = (size_t)lx * ly;
    uint32_t *stamp = (uint32_t *)calloc(N, sizeof(uint32_t));
    member_t *mb = (member_t *)malloc(sizeof(member_t) * (size_t)(9 * qx * qy + 8));
    view_t v = {&S, lat, (uint8_t *)lat, stamp, 1};
    int n = cell_members(&v, m % S.ncx, m / S.ncx, col, mb);
    for (int i = 0; i < n; i++) {
        origin[i] = sidx(&S, mb[i].ox, mb[i].oy);
        target[i] = sidx(&S, mb[i].tx, mb[i].ty);
        kind[i] = mb[i].kind;
        cls[i] = mb[i].cls;
    }
    free(stamp);
    free(mb);
    return n;
}

int orc_cell_writeset(int lx, int ly, int qx, int qy, int model, int m, int col,
                      int32_t *out)
{
    sys_t S;
    double r6[7] = {1, 1, 0, 1, 0.5, 1, 0};
    if (sys_init(&S, lx, ly, qx, qy, model, r6)) return -1;
    int *ws = (int *)malloc(sizeof(int) * (size_t)(qx * qy + 2 * (qx + qy) + 8));
    int n = cell_writeset(&S, m % S.ncx, m / S.ncx, col, ws);
    for (int i = 0; i < n; i++) out[i] = ws[i];
    free(ws);
    return n;
}

/*
 * Observables of Section 7 as exact integer sums: counts[s] = sites in
 * state s (s < 3); pairs = nearest-neighbour bonds (each once) with both
 * ends in state 1; gx[r-1], gy[r-1] = sum over sites of
 * [sigma(x)=1][sigma(x + r e)=1] along x and y, r = 1..rmax. A ring (ly = 1)
 * has no vertical bonds: its vertical terms are 0.
 */
void orc_observables(int lx, int ly, const uint8_t *lat, int rmax,
                     int64_t *counts, int64_t *pairs, int64_t *gx, int64_t *gy)
{
    counts[0] = counts[1] = counts[2] = 0;
    *pairs = 0;
    for (int r = 0; r < rmax; r++) gx[r] = gy[r] = 0;
    for (int y = 0; y < ly; y++)
        for (int x = 0; x < lx; x++) {
            int s = lat[(size_t)y * lx + x];
            if (s < 3) counts[s]++;
            if (s != 1) continue;
            *pairs += lat[(size_t)y * lx + (x + 1) % lx] == 1;
            if (ly > 1) *pairs += lat[(size_t)((y + 1) % ly) * lx + x] == 1;
            for (int r = 1; r <= rmax; r++) {
                gx[r - 1] += lat[(size_t)y * lx + (x + r) % lx] == 1;
                if (ly > 1) gy[r - 1] += lat[(size_t)((y + r) % ly) * lx + x] == 1;
            }
        }
}

/* M independent FS runs from the same initial state (replica r = 0..M-1,
 * window index from 0); final states into out[M*lx*ly]. */
int orc_fs_ensemble(int lx, int ly, int qx, int qy, int model,
                    const double *rates7, int scheme, double dt, double T,
                    uint64_t seed, int M, const uint8_t *init, uint8_t *out)
{
    size_t N = (size_t)lx * ly;
    for (int r = 0; r < M; r++) {
        uint8_t *lat = out + (size_t)r * N;
        uint32_t w = 0;
        uint64_t st[3] = {0, 0, 0};
        memcpy(lat, init, N);
        if (orc_fs_run(lx, ly, qx, qy, model, rates7, scheme, dt, T, seed,
                       (uint32_t)r, &w, 0, lat, st, NULL))
            return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The same FS run with the cells of each window spread over threads.       */
/* Same-colour cells read only the window-start snapshot outside their own  */
/* write sets and write disjoint write sets (Eq. exact), so the result does */
/* not depend on which thread runs which cell: it equals orc_fs_run's, bit  */
/* for bit. Each thread keeps its own private copy, stamps and member list; */
/* the snapshot is shared. Threads take cells from a shared counter.        */
/* ------------------------------------------------------------------------ */
typedef struct {
    const sys_t *S;
    uint8_t *lat, *snap;
    const int32_t *col;
    const double *hh;
    int64_t nw;
    uint32_t w0, rep;
    uint64_t seed;
    int32_t *workload;
    int *cells[2];
    int ncells[2];
    int next;
    pthread_barrier_t bar;
} tshared_t;

typedef struct {
    tshared_t *sh;
    work_t W;
    int tid;
    uint64_t ev, amb;
} tworker_t;

static void *thread_windows(void *arg)
{
    tworker_t *T = (tworker_t *)arg;
    tshared_t *sh = T->sh;
    const sys_t *S = sh->S;
    size_t N = (size_t)S->lx * S->ly;
    for (int64_t i = 0; i < sh->nw; i++) {
        const int c = sh->col[i];
        if (T->tid == 0) {
            memcpy(sh->snap, sh->lat, N);
            __atomic_store_n(&sh->next, 0, __ATOMIC_SEQ_CST);
        }
        pthread_barrier_wait(&sh->bar);
        for (;;) {
            int j = __atomic_fetch_add(&sh->next, 1, __ATOMIC_SEQ_CST);
            if (j >= sh->ncells[c]) break;
            int m = sh->cells[c][j];
            int a = 0;
            uint32_t e = cell_window(&T->W, sh->lat, m % S->ncx, m / S->ncx, c, sh->hh[i],
                                     sh->w0 + (uint32_t)i, sh->rep, sh->seed, &a);
            T->ev += e;
            T->amb += (uint64_t)a;
            if (sh->workload) sh->workload[m] = (int32_t)e;
        }
        pthread_barrier_wait(&sh->bar);
    }
    return NULL;
}

int orc_fs_run_threads(int lx, int ly, int qx, int qy, int model, const double *rates7,
                       int scheme, double dt, double T, uint64_t seed, uint32_t rep,
                       uint32_t *w, uint8_t *lat, uint64_t *stats_out, int32_t *workload,
                       int nthreads)
{
    sys_t S;
    if (nthreads < 1 || nthreads > 1024) return -1;
    if (!geometry_ok(model, lx, ly, qx, qy)) return -1;
    if (sys_init(&S, lx, ly, qx, qy, model, rates7)) return -1;
    int64_t nw = orc_schedule(scheme, dt, T, seed, rep, *w, NULL, NULL, 0);
    if (nw < 0) return -1;
    tshared_t sh;
    memset(&sh, 0, sizeof sh);
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nw + 1));
    double *hh = (double *)malloc(sizeof(double) * (size_t)(nw + 1));
    uint8_t *snap = (uint8_t *)malloc((size_t)lx * ly);
    int nc = S.ncx * S.ncy;
    sh.cells[0] = (int *)malloc(sizeof(int) * (size_t)nc);
    sh.cells[1] = (int *)malloc(sizeof(int) * (size_t)nc);
    tworker_t *tw = (tworker_t *)calloc((size_t)nthreads, sizeof(tworker_t));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int rc = -1, inited = 0;
    if (!col || !hh || !snap || !sh.cells[0] || !sh.cells[1] || !tw || !th) goto done;
    orc_schedule(scheme, dt, T, seed, rep, *w, col, hh, nw);
    for (int m = 0; m < nc; m++) {
        int c = ((m % S.ncx) + (m / S.ncx)) & 1;
        sh.cells[c][sh.ncells[c]++] = m;
    }
    sh.S = &S; sh.lat = lat; sh.snap = snap; sh.col = col; sh.hh = hh; sh.nw = nw;
    sh.w0 = *w; sh.rep = rep; sh.seed = seed; sh.workload = workload;
    for (; inited < nthreads; inited++) {
        tw[inited].sh = &sh;
        tw[inited].tid = inited;
        if (work_init(&tw[inited].W, &S)) { work_free(&tw[inited].W); goto done; }
        free(tw[inited].W.snap);
        tw[inited].W.snap = snap;   /* the shared window-start snapshot */
    }
    pthread_barrier_init(&sh.bar, NULL, (unsigned)nthreads);
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, thread_windows, &tw[t]);
    thread_windows(&tw[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
    pthread_barrier_destroy(&sh.bar);
    for (int t = 0; t < nthreads; t++) {
        stats_out[0] += tw[t].ev;
        stats_out[2] += tw[t].amb;
    }
    stats_out[1] += (uint64_t)nw;
    *w += (uint32_t)nw;
    rc = 0;
done:
    for (int t = 0; t < inited; t++) {
        tw[t].W.snap = NULL;
        work_free(&tw[t].W);
    }
    free(col); free(hh); free(snap); free(sh.cells[0]); free(sh.cells[1]); free(tw); free(th);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Nested (two-level) decomposition, Section 5 (Eq. sublatt2, Eq. opdecomp2)*/
/* The lattice is a checkerboard of super-cells Qx*Qy (colours E/O, as in   */
/* Eq. sublatt); every super-cell is itself a checkerboard of sub-cells     */
/* qx*qy (Eq. sublatt2), so L^E_m = L^EE_m + L^EO_m. The outer schedule     */
/* (Lie, Strang, random) runs over the super-cell colours with step dt as   */
/* in orc_fs_run; within an outer window of colour C and length h every     */
/* super-cell of colour C runs the inner schedule over its sub-cell colours */
/* with n_in inner steps of length h/n_in: inner Lie  EE(d) EO(d), inner    */
/* Strang EE(d/2) EO(d) EE(d/2) per inner step. Every inner window is an FS */
/* window of the sub-cells of one inner colour inside the super-cells of    */
/* colour C (the sub-cell checkerboard of a super-cell is the global one    */
/* since Qx/qx and Qy/qy are even), reading the lattice as it was when the  */
/* inner window began. Spin-flip models only: there every event is a site   */
/* event, so both levels of the decomposition are the site partition.       */
/* Draws: the inner window j of outer window W uses window index            */
/* W * ninner + j (ninner = 2 n_in for inner Lie, 3 n_in for inner Strang)  */
/* and the sub-cell's id in the global sub-cell grid.                       */
/* stats_out = {events, inner windows, ambiguous}; *w counts outer windows. */
/* ------------------------------------------------------------------------ */
static int nested_ok(int model, int lx, int ly, int Qx, int Qy, int qx, int qy, int inner, int n_in)
{
    if (model != ORC_ADSDES && model != ORC_ISING) return 0;
    if (inner != ORC_LIE && inner != ORC_STRANG) return 0;
    if (n_in < 1) return 0;
    if (qx < 1 || qy < 1 || Qx < 2 * qx || Qy < 2 * qy) return 0;
    if (Qx % (2 * qx) || Qy % (2 * qy)) return 0;
    if (lx < 2 * Qx || ly < 2 * Qy || lx % (2 * Qx) || ly % (2 * Qy)) return 0;
    return geometry_ok(model, lx, ly, qx, qy);
}

int orc_fs2_run(int lx, int ly, int Qx, int Qy, int qx, int qy, int model,
                const double *rates7, int scheme, double dt, double T, int inner, int n_in,
                uint64_t seed, uint32_t rep, uint32_t *w, uint8_t *lat, uint64_t *stats_out,
                int32_t *workload)
{
    sys_t S;
    if (!nested_ok(model, lx, ly, Qx, Qy, qx, qy, inner, n_in)) return -1;
    if (sys_init(&S, lx, ly, qx, qy, model, rates7)) return -1;
    int64_t nw = orc_schedule(scheme, dt, T, seed, rep, *w, NULL, NULL, 0);
    if (nw < 0) return -1;
    const int64_t ninner = (inner == ORC_LIE ? 2 : 3) * (int64_t)n_in;
    if (((int64_t)*w + nw) * ninner > (int64_t)UINT32_MAX) return -1;
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nw + 1));
    double *hh = (double *)malloc(sizeof(double) * (size_t)(nw + 1));
    work_t W;
    memset(&W, 0, sizeof W);
    if (!col || !hh || work_init(&W, &S)) { work_free(&W); free(col); free(hh); return -1; }
    orc_schedule(scheme, dt, T, seed, rep, *w, col, hh, nw);
    const size_t N = (size_t)lx * ly;
    const int rx = Qx / qx, ry = Qy / qy;   /* sub-cells per super-cell side */
    uint64_t ev = 0, amb = 0;
    for (int64_t i = 0; i < nw; i++) {
        const int C = col[i];
        const double d = hh[i] / (double)n_in;
        const uint32_t W0 = (uint32_t)((*w + (uint32_t)i) * ninner);
        for (int64_t j = 0; j < ninner; j++) {
            int cin;
            double len;
            if (inner == ORC_LIE) { cin = (int)(j % 2); len = d; }
            else { int p = (int)(j % 3); cin = p == 1; len = p == 1 ? d : d * 0.5; }
            memcpy(W.snap, lat, N);
            for (int m = 0; m < S.ncx * S.ncy; m++) {
                const int sx = m % S.ncx, sy = m / S.ncx;
                if (((sx + sy) & 1) != cin) continue;
                if ((((sx / rx) + (sy / ry)) & 1) != C) continue;
                int a = 0;
                uint32_t e = cell_window(&W, lat, sx, sy, cin, len, W0 + (uint32_t)j, rep, seed, &a);
                ev += e;
                amb += (uint64_t)a;
                if (workload) workload[m] = (int32_t)e;
            }
        }
    }
    *w += (uint32_t)nw;
    stats_out[0] += ev;
    stats_out[1] += (uint64_t)(nw * ninner);
    stats_out[2] += amb;
    work_free(&W);
    free(col);
    free(hh);
    return 0;
}

/* M independent nested runs (replicas 0..M-1) from the same initial state. */
int orc_fs2_ensemble(int lx, int ly, int Qx, int Qy, int qx, int qy, int model,
                     const double *rates7, int scheme, double dt, double T, int inner,
                     int n_in, uint64_t seed, int M, const uint8_t *init, uint8_t *out)
{
    size_t N = (size_t)lx * ly;
    for (int r = 0; r < M; r++) {
        uint8_t *lat = out + (size_t)r * N;
        uint32_t w = 0;
        uint64_t st[3] = {0, 0, 0};
        memcpy(lat, init, N);
        if (orc_fs2_run(lx, ly, Qx, Qy, qx, qy, model, rates7, scheme, dt, T, inner, n_in,
                        seed, (uint32_t)r, &w, lat, st, NULL))
            return -1;
    }
    return 0;
}

/* M independent serial SSA runs from the same initial state. */
int orc_ssa_ensemble(int lx, int ly, int model, const double *rates7, double T,
                     uint64_t seed, int M, const uint8_t *init, uint8_t *out)
{
    size_t N = (size_t)lx * ly;
    for (int r = 0; r < M; r++) {
        uint8_t *lat = out + (size_t)r * N;
        memcpy(lat, init, N);
        if (orc_ssa_run(lx, ly, model, rates7, T, seed, (uint32_t)r, lat) < 0)
            return -1;
    }
    return 0;
}

/* One window of colour col for the listed cells only (the sampled check of
 * full-size lattices): every listed cell must have colour col; each runs
 * against the lattice as it was when the window began and writes its write
 * set into lat. events[i] receives cell cells[i]'s event count and amb[i]
 * its ambiguity flag. Returns 0, or -1 on invalid arguments. */
int orc_window_cells(int lx, int ly, int qx, int qy, int model,
                     const double *rates7, int col, double h, uint32_t w,
                     uint64_t seed, uint32_t rep, uint8_t *lat, int ncells,
                     const int32_t *cells, int32_t *events, int32_t *amb)
{
    sys_t S;
    if (!geometry_ok(model, lx, ly, qx, qy)) return -1;
    if (sys_init(&S, lx, ly, qx, qy, model, rates7)) return -1;
    for (int i = 0; i < ncells; i++) {
        int m = cells[i];
        if (m < 0 || m >= S.ncx * S.ncy) return -1;
        if ((((m % S.ncx) + (m / S.ncx)) & 1) != col) return -1;
    }
    work_t W;
    if (work_init(&W, &S)) { work_free(&W); return -1; }
    memcpy(W.snap, lat, (size_t)lx * ly);
    for (int i = 0; i < ncells; i++) {
        int m = cells[i], a = 0;
        events[i] = (int32_t)cell_window(&W, lat, m % S.ncx, m / S.ncx, col, h, w, rep,
                                         seed, &a);
        amb[i] = a;
    }
    work_free(&W);
    return 0;
}
