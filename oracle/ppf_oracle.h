/*
 * ppf_oracle.h -- declarations of the FP64 CPU oracle (test infrastructure
 * only; the CUDA library never includes this header).
 */
#ifndef PPF_ORACLE_H
#define PPF_ORACLE_H
#include <stdint.h>

enum { ORC_OK = 0, ORC_EDEGENERATE = 5, ORC_EINTERNAL = 7 };
enum { ORC_SYSTEMATIC = 0, ORC_RPA_GS = 1, ORC_RPA_SGS = 2, ORC_RPA_LGS = 3, ORC_RNA = 4,
       ORC_RPA2_GS = 5, ORC_RPA2_SGS = 6, ORC_RPA2_LGS = 7, ORC_ARNA = 8 };
enum { ORC_PURPOSE_INIT = 0, ORC_PURPOSE_PROP = 1, ORC_PURPOSE_RESAMPLE = 2,
       ORC_PURPOSE_GROUP_RESAMPLE = 3, ORC_PURPOSE_RING = 4 };

typedef struct {
    int32_t width, height, patch_radius;
    int32_t likelihood; /* 0: eq. 4 at the particle; 1: piecewise constant over pixel cells (pcSIR) */
    double psf_sigma, amplitude, background, sigma_xi;
    double sigma_m, sigma_v, sigma_I, v0_max;
    uint64_t seed;
    uint32_t filter_id, pad2_;
} orc_model;

int orc_set_threads(int n);
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u01(uint32_t r);
double orc_u21(uint32_t field);
void orc_prop_fields(const uint32_t r[4], uint32_t f[6]);
void orc_normals5(uint64_t seed, uint32_t slot, uint32_t frame, uint32_t filter, double e[5]);
void orc_init(const orc_model *m, int64_t N, double *st);
void orc_propagate(const orc_model *m, int64_t N, int32_t frame, const double *par,
                   const int32_t *anc, const double *lw_prev, double *st);
void orc_propagate_slots(const orc_model *m, int64_t n, int32_t frame, const int64_t *slots,
                         const double *parents5, double *out5);
void orc_loglik_many(const orc_model *m, const double *frame, int64_t n, const double *x, const double *y,
                     const double *I0, double *l);
double orc_loglik(const orc_model *m, const double *frame, double x, double y, double I0);
void orc_weight(const orc_model *m, int64_t N, const double *frame, double *st);
void orc_summary(int64_t N, const double *st, const double *lw_prev, double out[8]);
int orc_scale_bits(int64_t n);
float orc_exp2_frac(float f);
uint64_t orc_quantise(float lw, float M, int s);
int64_t orc_tickets_below(uint64_t c, int64_t n, uint64_t u, uint64_t Q);
uint64_t orc_ticket_offset(uint64_t seed, uint32_t filter, uint32_t frame, uint32_t purpose,
                           uint32_t index, uint64_t Q);
int orc_systematic(int64_t n_in, const uint64_t *q, int64_t n_tickets, uint64_t u,
                   int64_t base, int32_t *anc_out, int64_t *offspring);
int64_t orc_schedule(int scheme, int32_t G, const int64_t *count, const int64_t *target,
                     int32_t *src, int32_t *dst, int64_t *cnt);
void orc_balanced_offsets(int64_t N, int32_t G, int64_t *off);
int orc_resample(const orc_model *m, int scheme, double alpha, int64_t N, int32_t frame,
                 int32_t G, const int64_t *goff_in, const float *lw, const double *lw_sum,
                 int32_t *anc, double *lw_reset, int64_t *goff_out, int64_t stats[4]);
void orc_arna_ring(uint64_t seed, uint32_t filter, uint32_t frame, int32_t G, int32_t *ring);
int orc_resample_arna(const orc_model *m, double alpha, int64_t N, int32_t frame, int32_t G,
                      const int64_t *goff_in, const float *lw, const double *lw_sum, int32_t lost,
                      int32_t *ring, int32_t *anc, double *lw_reset, int64_t *goff_out, int64_t stats[5]);
int orc_run(const orc_model *m, int64_t N, int32_t group_size, int scheme, double alpha,
            double ess_threshold, int32_t K, const double *frames, double *est, double *st_out);
void orc_loglik_partials(const orc_model *m, const double *frame, double x, double y, double I0, int32_t ax,
                         int32_t ay, double out[6]);
int orc_grad_run(const orc_model *m0, int64_t N, int32_t K, const double *frames, const double theta[4],
                 int replay, int32_t *anc_io, int32_t *anchor_io, double *L_out, double grad[4]);
#endif
