// The hopping stencil H_{p,1-p} (Eq. 4) and the kernels built on it:
//   M_HOP   out = H in                       (qcd_dslash_eo)
//   M_MULT  out = F^-1 H in                  (MULT = H~, Sec. II-B)
//   M_DHAT  out = a*y + cc*F^-1 H in + d*z   (second half of D^ = 1 - k^2 H~_eo H~_oe,
//                                             with the dot products of Alg. 2 fused)
//   M_SRC   out = F^-1 (a*y + cc*H in)       (b^_e, Eq. 6, and x_o, Eq. 7)
//   M_FULL  out = a*F y + cc*H in + d*z      (D = F - kappa H on one parity, residuals)
//   M_RECON out = F^-1 (a*y + cc*H in) and |a*y + cc*H in - F out|^2 (FP64 only)
//
// One thread computes one output site (and one right-hand side: the
// right-hand sides of a site sit in the same block so that its links and
// clover entries are fetched from HBM once and hit L1 for the others).
// For each of the 8 directions the neighbour spinor is projected with
// (1 -/+ gamma_mu) to two spin components before the colour multiply
// (the rank-2 structure of Eq. 4), the link is rebuilt from 12 reals for
// FP32/FP16 (Sec. III-A), multiplied, and expanded back.
#include "stencil.cuh"

namespace qcd {

// per-precision instantiations (stencil_<prec>.cu) and the multi-RHS kernel
int dispatch_f64(const StencilCall &sc, const StencilArgs &A, dim3 grid, dim3 block, cudaStream_t s, int v);
int dispatch_f32(const StencilCall &sc, const StencilArgs &A, dim3 grid, dim3 block, cudaStream_t s, int v);
int dispatch_f32_rg(const StencilCall &sc, const StencilArgs &A, int bx, cudaStream_t s, int v);
int dispatch_f16(const StencilCall &sc, const StencilArgs &A, dim3 grid, dim3 block, cudaStream_t s, int v);
int dispatch_df64(const StencilCall &sc, const StencilArgs &A, dim3 grid, dim3 block, cudaStream_t s, int v);
int launch_mrhs(const StencilCall &sc, const StencilArgs &A, int nrhs, cudaStream_t s, int variant, int tile,
                int num_sms);

// Algorithmic bytes per output site of one stencil launch (each input read
// once, the output written once), by precision: spinor, link, clover.
static void site_bytes(int prec, double &spinor, double &link, double &clover)
{
    if (prec == QCD_F64 || prec == QCD_DF64) { spinor = 192; link = 144; clover = 576; }
    else if (prec == QCD_F32) { spinor = 96; link = 48; clover = 288; }
    else { spinor = 52; link = 24; clover = 144; }
}

unsigned tune_key(const StencilCall &sc)
{
    const unsigned nr = sc.nrhs < 1 ? 1 : (sc.nrhs > 31 ? 31 : sc.nrhs);
    return (unsigned)sc.prec | ((unsigned)sc.mode << 2) | ((unsigned)sc.red << 5) | ((unsigned)(sc.dagger != 0) << 7) |
           (nr << 8);
}

double stencil_bytes(const qcd_ctx *c, const StencilCall &sc)
{
    double sp, lk, cl;
    site_bytes(sc.prec, sp, lk, cl);
    const int nrhs = sc.nrhs < 1 ? 1 : sc.nrhs;
    double per_site = nrhs * 2 * sp + 8 * lk;  // in, out, links
    if (sc.mode != M_HOP) per_site += cl;
    if (sc.mode == M_DHAT || sc.mode == M_SRC || sc.mode == M_FULL || sc.mode == M_RECON) per_site += nrhs * sp;  // y
    if (sc.mode == M_RECON) per_site += cl;  // F as well as F^-1
    if (sc.d != 0.0 && (sc.mode == M_DHAT || sc.mode == M_FULL)) per_site += nrhs * sp;   // z
    if (sc.red == R_DOT_AUX || (sc.red == R_OMEGA && sc.aux.p != sc.y.p)) per_site += nrhs * sp;
    return per_site * c->g.Vh;
}

bool is_mrhs(const StencilCall &sc)
{
    return sc.prec == QCD_F32 && sc.nrhs > 1 && sc.red == R_NONE && (sc.mode == M_MULT || sc.mode == M_HOP);
}

int launch_stencil(qcd_ctx *c, const StencilCall &sc)
{
    StencilArgs A;
    A.g = c->g;
    const int p = sc.prec;
    for (int par = 0; par < 2; ++par) {
        A.U.a[par] = p == QCD_F64 ? c->U64[par] : p == QCD_F32 ? c->U32[par] : p == QCD_DF64 ? c->UDF[par] : c->U16a[par];
        A.U.b[par] = c->U16b[par];
        A.C.p[par] = (sc.mode == M_FULL) ? c->C[p][par] : c->Ci[p][par];
        A.Cf.p[par] = c->C[p][par];
    }
    A.out = sc.out.sp();
    A.in = sc.in.sp();
    A.y = sc.y.sp();
    A.aux = sc.aux.sp();
    A.z = sc.z.sp();
    A.out_par = sc.out_par;
    A.a = sc.a;
    A.cc = sc.cc;
    A.d = sc.d;
    A.af = (float)sc.a;
    A.ccf = (float)sc.cc;
    A.df32 = (float)sc.d;
    A.has_z = sc.d != 0.0;
    A.rhs_stride = sc.rhs_stride;
    A.norm_stride = sc.norm_stride;
    A.nrhs = sc.nrhs < 1 ? 1 : sc.nrhs;
    A.red = sc.red_args;
    A.done = sc.done;
    A.done_stride = sc.done_stride;
    A.red_pstride = sc.red_pstride;
    A.skip = nullptr;
    const int nrhs = sc.nrhs < 1 ? 1 : sc.nrhs;
    if (nrhs > 16) {
        set_error_message("nrhs > 16 per launch");
        return QCD_EINVAL;
    }
    if (sc.rhs_grid) {
        // a lockstep second half: the single-RHS entry's register budget and
        // sites per block, so that every right-hand side repeats the
        // single-RHS launch's arithmetic and reduction order
        if (p != QCD_F32 || sc.mode != M_DHAT || (sc.red != R_DOT_AUX && sc.red != R_OMEGA) ||
            sc.done_stride < 1 || !sc.red_pstride) {
            set_error_message("rhs_grid: FP32 D^ second halves with per-RHS states and partials only");
            return QCD_EINVAL;
        }
        StencilCall one = sc;
        one.nrhs = 1;
        one.rhs_grid = false;
        int v = 0, b = 128;
        auto it = c->tune.find(tune_key(one));
        if (it != c->tune.end()) {
            v = it->second.variant;
            b = it->second.bx;
        }
        if (v != 1) v = 0;  // the rolled and pipelined hops have no lockstep form: the plain kernel
        if ((size_t)nblocks(c->g.Vh, b) * 4 > sc.red_pstride) {
            set_error_message("rhs_grid: %u partials per right-hand side do not fit", nblocks(c->g.Vh, b));
            return QCD_EINVAL;
        }
        const int rc = dispatch_f32_rg(sc, A, b, c->stream, v);
        if (rc != QCD_OK) return rc;
        c->launches += 1;
        QCD_CUDA_CHECK(cudaGetLastError());
        return QCD_OK;
    }
    int bx = 128, variant = 0;  // bx: sites per block, or for the multi-RHS kernel the RHS tile
    if (nrhs > 1) bx = is_mrhs(sc) ? nrhs : nrhs <= 4 ? 64 : 32;
    if (sc.force_variant >= 0) {
        variant = sc.force_variant;
        bx = sc.force_bx;
    } else {
        auto it = c->tune.find(tune_key(sc));
        if (it != c->tune.end()) {
            variant = it->second.variant;
            bx = it->second.bx;
        }
    }
    if (!is_mrhs(sc) && bx * nrhs > 384) {
        // more right-hand sides than a block of the generic kernels holds:
        // launch them in groups (no reduction spans the groups)
        if (sc.red != R_NONE) {
            set_error_message("a fused reduction over %d right-hand sides is not supported", nrhs);
            return QCD_EINVAL;
        }
        const int per = 384 / bx;
        for (int r0 = 0; r0 < nrhs; r0 += per) {
            StencilCall g = sc;
            g.nrhs = nrhs - r0 < per ? nrhs - r0 : per;
            g.force_variant = variant;
            g.force_bx = bx;
            HVec *vs[5] = {&g.out, &g.in, &g.y, &g.z, &g.aux};
            for (HVec *v : vs) {
                if (v->p) v->p = (char *)v->p + (size_t)r0 * sc.rhs_stride * 16;
                if (v->norm) v->norm += (size_t)r0 * sc.norm_stride;
            }
            const int rc = launch_stencil(c, g);
            if (rc != QCD_OK) return rc;
        }
        return QCD_OK;
    }
    dim3 block(bx, nrhs);
    dim3 grid(nblocks(c->g.Vh, bx));
    if (!is_mrhs(sc) && sc.red != R_NONE && (int)grid.x > c->partial_blocks) {
        set_error_message("reduction grid too large");
        return QCD_EINVAL;
    }
    // the second half of an even-odd operator with its fused dots (D^_ee:
    // M_DHAT; S_ee: M_FULL with a reduction) is timed apart from the MULTs
    const bool second_half = sc.mode == M_DHAT || (sc.mode == M_FULL && sc.red != R_NONE);
    const int cls = p == QCD_F32    ? (second_half ? QCD_K_DHAT_F32 : QCD_K_MULT_F32)
                    : p == QCD_F16  ? QCD_K_MULT_F16
                    : p == QCD_DF64 ? QCD_K_MULT_DF64
                                    : QCD_K_MULT_F64;
    ProfScope prof(c, cls, stencil_bytes(c, sc));
    A.skip = prof.flag;
    int rc;
    const int rv = variant;
    if (is_mrhs(sc)) rc = launch_mrhs(sc, A, nrhs, c->stream, rv, bx, c->num_sms);
    else if (p == QCD_F64) rc = dispatch_f64(sc, A, grid, block, c->stream, rv);
    else if (p == QCD_F32) rc = dispatch_f32(sc, A, grid, block, c->stream, rv);
    else if (p == QCD_DF64) rc = dispatch_df64(sc, A, grid, block, c->stream, rv);
    else rc = dispatch_f16(sc, A, grid, block, c->stream, rv);
    if (rc != QCD_OK) return rc;
    QCD_CUDA_CHECK(cudaGetLastError());
    return QCD_OK;
}

}  // namespace qcd
