/*
 * fse_oracle.h -- FP64 CPU oracle for FSE block concealment.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the product library.
 */
#ifndef FSE_ORACLE_H
#define FSE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Sample classes of the extrapolation area (Sec. 2, Fig. 1). */
enum {
    ORACLE_CLS_A = 0,   /* originally known sample (support area A)        */
    ORACLE_CLS_R = 1,   /* lost sample concealed earlier (area R)          */
    ORACLE_CLS_BI = 2,  /* lost sample inside the processed block (B_i)    */
    ORACLE_CLS_BO = 3,  /* lost sample outside the block, still open (B_o) */
    ORACLE_CLS_OUT = 4  /* position outside the image                      */
};

/* Processing order.  order 0 = line scan (Sec. 2), 1 = Algorithm 1 (Sec. 3).
 * lost: [bh*bw] block-loss flags, row-major.  Outputs (caller-owned):
 * group_of_block [bh*bw] (-1 = nothing to do), group_ptr [groups+1],
 * block_ids [lost blocks] listing each group in scan order.
 * Returns 0, or a negative value on bad arguments / allocation failure. */
int oracle_plan(int bw, int bh, const uint8_t *lost, int order,
                int32_t *group_of_block, int32_t *group_ptr,
                int32_t *block_ids, int32_t *n_groups);

/* Eq. (2) weighting over an M x N area with per-sample classes. */
void oracle_weights(int M, int N, const uint8_t *cls, double rho, double delta,
                    double *w);

/* FSE of one M x N area with an F x F DFT basis and K iterations.
 * f, cls: [M*N] row-major.  want_g (optional): which g samples to evaluate.
 * Optional outputs (NULL to skip): g_out [M*N] real part of the model,
 * w_out [M*N], R0_out/W_out/R_out/coef_out [F*F complex interleaved],
 * u_out [K] selected linear index F*k_m + k_n, dc_out [K complex],
 * margin_out [K]: per iteration, |R_w[u]| minus the largest |R_w[k]| over
 * k != u, divided by sum|w f| + W[0] * sum of the earlier |dc| (HUGE_VAL
 * when there is no competitor or no support); an exact tie gives 0, except
 * an exact tie with the conjugate partner k = -u, which is skipped. */
int oracle_extrapolate_area(int M, int N, int F, const double *f,
                            const uint8_t *cls, double rho, double delta,
                            double gamma, int K, int tie_largest,
                            const uint8_t *want_g, double *g_out,
                            double *w_out, double *R0_out, double *W_out,
                            int32_t *u_out, double *dc_out, double *R_out,
                            double *coef_out, double *margin_out);

/* Whole frame.  img, mask: [H*Wd] uint8 (mask 1 = lost sample).  Block size
 * B, border d (area M = B + 2d <= F).  threads: OpenMP threads over the
 * blocks of a group.  work [H*Wd] FP64 working frame, out [H*Wd] uint8,
 * group_of_block_out [bh*bw] (optional), u_trace [bh*bw][K] (optional): the
 * selected indices of every concealed block (rows of other blocks are left
 * untouched). */
int oracle_conceal_frame(int H, int Wd, const uint8_t *img,
                         const uint8_t *mask, int B, int d, int F, int K,
                         double rho, double delta, double gamma, int order,
                         int threads, double *work, uint8_t *out,
                         int32_t *group_of_block_out, int32_t *u_trace);

/* As oracle_conceal_frame, plus (optional) cls_trace [bh*bw][M*M]: the
 * sub-area class of every area sample of each concealed block as its group
 * saw the frame (ORACLE_CLS_*; rows of other blocks are left untouched), and
 * margin_trace [bh*bw][K]: the selection margins of each concealed block
 * (see oracle_extrapolate_area). */
int oracle_conceal_frame_ex(int H, int Wd, const uint8_t *img,
                            const uint8_t *mask, int B, int d, int F, int K,
                            double rho, double delta, double gamma, int order,
                            int threads, double *work, uint8_t *out,
                            int32_t *group_of_block_out, int32_t *u_trace,
                            uint8_t *cls_trace, double *margin_trace);

int oracle_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
