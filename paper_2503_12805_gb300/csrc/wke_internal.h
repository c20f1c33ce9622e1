// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <string>
#include <vector>

#include "wke.h"

namespace wke {

// Thread-local error message for wke_last_error_string().
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);

// ---------------------------------------------------------------- host plan
// Quadrature nodes and the field / product layout of one plan, all in double
// precision on the host (Sec. 3.3, Eq. (3.8)).
struct HostPlan {
    int d = 0, N = 0, M = 0;
    // N is the grid of the transforms; N_in the grid of f and Q.  They differ
    // only for de-aliased plans (N = 2 N_in, zero padding).
    int N_in = 0;
    bool dealias = false;
    // WKE_SPLIT: precision is WKE_FP32 (float data) and the axis-0
    // transforms use the tensor-core DFT
    bool split = false;
    double L = 0, R = 0;
    int n_r = 0, n_s = 0, n_sig = 0;
    int precision = WKE_FP64, nyquist = WKE_NYQ_KEEP, dispersion = WKE_OMEGA_HALF_K2;

    std::vector<double> r, w_r;          // radial nodes / weights on [0, R]
    std::vector<double> qhat, w_s;       // n_s * d directions, weights
    std::vector<double> sig, w_sig;      // n_sig * d collision angles, weights

    // Per node p = (p1, p2, p3) in lexicographic order.
    std::vector<double> W;               // w_r |q|^{2d-3} w_s w_sig
    std::vector<double> q, a, b;         // shift vectors, M * d each

    // Field layout.  Group g = p1 * n_s + p2 owns fields_per_group shifted
    // fields f_N(k - x): local field 0 is C (x = q); with antipodal pairing
    // local field 1 + p3 is f_N(k - a_{p3}) (which is also f_N(k - b) of the
    // antipodal node), otherwise 1 + 2 p3 is A_{p3} and 2 + 2 p3 is B_{p3}.
    bool paired = false;
    std::vector<int> anti;               // sigma index of -sigma (paired only)
    int fields_per_group = 0, products_per_group = 0, n_groups = 0;
    std::vector<double> field_shift;     // n_groups * fields_per_group * d
    std::vector<int> prod_fa, prod_fb;   // n_groups * products_per_group local field ids
    std::vector<double> prod_W;          // n_groups * products_per_group weights

    // Chunking of groups through the intermediate buffer.  Pass 1 transforms
    // "units": two shifted fields packed as one complex transform of
    // ghat (E_a + i E_b).  A chunk of ng groups has ceil(ng / 2) C units (the
    // C fields of groups 2k and 2k+1 together; a lone C when ng is odd)
    // followed by ng * products_per_group product units (fields fa, fb of
    // each product).
    int groups_per_chunk = 0, n_chunks = 0;
    size_t chunk_bytes = 0;

    // Shared-field layout (`shared`): a chunk is a run of groups and the
    // distinct shifted fields they need (fields with the same shift vector,
    // e.g. the C field of one direction and an A field of another, are one
    // field); each distinct field is transformed once per evaluation.  Units
    // pack the chunk's fields in order (fields 2u, 2u + 1).  Pass 2
    // transforms the units along axis 0 in place and a product pass reads
    // every field of the chunk at each point.  In this layout field_shift
    // lists the distinct fields of all chunks, prod_fa / prod_fb hold
    // chunk-local field ids and group_cfield the chunk-local id of each
    // group's C field.
    bool shared = false;
    std::vector<int> chunk_g0, chunk_f0;  // n_chunks + 1 entries: first group, first field
    std::vector<int> group_cfield;        // n_groups
    int max_chunk_fields = 0;
    int n_fields_total = 0;               // rows of the phase table

    // Separable transforms (3D, shared-field layout).  The phase of a field
    // with shift x factors per axis, exp(-i pi j.x / L) = E0(j1, x0) E1(j2, x1)
    // E2(j3, x2), so the inverse transform of ghat E_x over axis 2 depends on
    // x2 alone and the one over axes 1 and 2 on (x1, x2) alone; only the
    // axis-0 transform is per field.  Per chunk the distinct x2 values
    // ("row values") and the distinct (x1, x2) pairs are listed, the pairs
    // grouped by row value; the trailing-axis pass transforms each row value
    // and each pair once per plane, and each unit's axis-0 transform starts
    // from the pair planes of its two fields.
    bool separable = false;
    std::vector<int> chunk_v0, chunk_p0;  // n_chunks + 1: first row value / first pair of each chunk
    std::vector<int> sep_v;               // per row value: a field with that x2 (global id), first
                                          // and end pair (chunk-local), 3 ints each
    std::vector<int> sep_p;               // per pair: a field with that (x1, x2) (global id)
    std::vector<int> field_pair;          // per field: its pair (chunk-local)
    int max_chunk_pairs = 0, max_chunk_values = 0;
    std::vector<int> chunk_u0;            // n_chunks + 1: first unit of each chunk (shared layout)
    // The product pass of the shared layout fused with the axis-0 transform
    // (3D, FP32, not split): no unit buffer between them.  can_fuse is the
    // capability, fused the current choice (wke_tuning.fuse_products).
    bool can_fuse = false;
    // The cube rule's own product schedule for the fused kernel (3D N = 64,
    // shared layout, cube q-hat and sigma rules with antipodal pairing): in every
    // chunk the fields are the 26 shifts m s, s in {-1, 0, 1}^3 \ {0}; group
    // v (a vertex, s = v, its C field) has the three products (edge field of
    // axis i with sign v_i, face field with component i zero and the other
    // signs of v), i = 0, 1, 2.  Per chunk, chunk-local field ids of the edge
    // fields (index 2 i + [sign < 0]), the face fields (index 4 i + q, bit 0 of
    // q: the lower other axis negative, bit 1: the higher one) and the C
    // fields, and the group weights, both by vertex (bit a: v_a < 0).  Empty
    // unless every chunk has this form.
    struct CubeChunk {
        int edge[6], face[12], cfield[8];
        double w[8];
    };
    std::vector<CubeChunk> cube;
    bool tune_rule_products = true;      // use `cube` where present (wke_tuning.rule_products)
    bool fused = false;

    double scale = 0;                    // 2^{1-d} (times 1/2 for omega = |k|^2)

    // Launch layout (wke_plan_set_tuning / wke_plan_autotune).
    int tune_p2_points = 8;              // pass-2 points per thread (4 or 8; N >= 128 uses 8)
    int tune_p1_units_per_block = 0;     // pass-1 units per block (0 = automatic: 2 shared, 3 per-group)
    bool tune_forward_fp32 = false;      // FP32 plans: the forward transform in float (default double)
};

// Validate arguments and fill `hp` (no device work).  Returns WKE_OK or an
// error code with the message set.
int build_host_plan(int d, int N, double L, int M, const wke_quadrature *quad, HostPlan &hp);

// exp(-i pi j x / L) for the signed mode j stored at DFT position `pos`.
void phase_row(int N, double L, double x, double *out_re_im /* 2N */);

// Device bytes of every buffer a plan with this layout allocates.
size_t plan_device_bytes(const HostPlan &hp);

// Arithmetic and intermediate-traffic model of one collision (for info).
double plan_flops(const HostPlan &hp);
double plan_l2_bytes(const HostPlan &hp);
double total_units(const HostPlan &hp);

// ---------------------------------------------------------------- kernels
// Launch wrappers (wke_kernels_*.cu).  All are asynchronous on `stream`;
// they return cudaGetLastError() cast to int.
struct DevicePtrs {
    // Set by the API layer; element types depend on the precision.
    const void *f;            // input grid (T)
    void *ghat;               // N^d complex T: coefficients of f (DFT order)
    void *fwd_tmp;            // N^d complex double: forward-transform scratch
    void *H;                  // chunk intermediate units, complex T
    void *V;                  // chunk Nyquist tables: per unit, d tables of N^{d-1} (V_a, V_b) pairs
    void *nslice;             // d masked Nyquist slices of ghat, N^{d-1} complex T each
    double *Qacc;             // groups_per_chunk * N^d partial sums (real)
    double *Qacc_im;          // groups_per_chunk * N^d partial sums (imag) or null
    const void *phase;        // n_fields * d * N complex T phase tables
    const void *tw;           // N complex T twiddles exp(+2 pi i k / N)
    const double *tw64;       // N_in complex double twiddles (forward transform of f)
    // de-aliased plans only
    void *ghat_in;            // N_in^d complex T: coefficients of f on its own grid
    void *ffine;              // N^d T: f_N on the 2N grid (F in the products)
    void *map0, *map1;        // N^d complex double each: per-axis map buffers
    const void *Kint;         // N x N_in complex double: values on the 2N grid from the N_in grid
    const void *Kproj;        // N_in x N complex double: projection onto modes [-N_in/2, N_in/2-1]
    const int *prod_local;    // n_groups * products_per_group * 2 ints: local fields (fa, fb)
    const int *group_cfield;  // shared-field layout: chunk-local C field of each group
    // separable transforms
    void *S;                  // chunk pair planes: max_chunk_pairs * N^3 complex T
    const int *sep_v;         // 3 ints per row value (HostPlan::sep_v)
    const int *sep_p;         // per pair: field for the axis-1 phase row
    const int *field_pair;    // per field: chunk-local pair
    const void *unit_e0;      // FP32 separable: per unit and j1, (E0(j1, x0a), E0(j1, x0b)) as float4
                              // (zero second part for a lone field)
    // fused product kernel, last chunk of an evaluation: write Q (and Im Q)
    // = scale_out * accumulator and clear the accumulators (null otherwise)
    void *Qout, *Qiout;
    double scale_out;
    const double *prod_W;     // n_groups * products_per_group
};

// Units of a chunk of ng groups (C units first, then product units).
inline int chunk_units(const HostPlan &hp, int ng) { return (ng + 1) / 2 + ng * hp.products_per_group; }
// Units of chunk c in either layout; the most units any chunk has.
inline int units_of_chunk(const HostPlan &hp, int c) {
    if (hp.shared) return (hp.chunk_f0[c + 1] - hp.chunk_f0[c] + 1) / 2;
    const int g0 = c * hp.groups_per_chunk;
    return chunk_units(hp, hp.groups_per_chunk < hp.n_groups - g0 ? hp.groups_per_chunk : hp.n_groups - g0);
}
// FP64 accumulators of N^d points: one per group of a chunk (per-group
// layout) or one in all (shared-field layout)
inline int n_accumulators(const HostPlan &hp) { return hp.shared ? 1 : hp.groups_per_chunk; }
inline int max_chunk_units(const HostPlan &hp) {
    return hp.shared ? (hp.max_chunk_fields + 1) / 2 : chunk_units(hp, hp.groups_per_chunk);
}
size_t chunk_unit_bytes(const HostPlan &hp);   // H buffer bytes for a full chunk
size_t chunk_v_bytes(const HostPlan &hp);      // V buffer bytes for a full chunk
size_t chunk_s_bytes(const HostPlan &hp);      // S buffer bytes for a full chunk (separable plans)
int launches_per_collision(const HostPlan &hp);
// The unit buffers H: the output of pass 1 (per-unit transforms) or of the
// separate axis-0 pass; a separable plan whose axis-0 transform is fused
// with the products has none.
inline bool needs_unit_buffers(const HostPlan &hp) { return !(hp.separable && hp.fused); }
// Dynamic shared memory of the fused axis-0 + product kernel (3D FP32).
size_t fused_smem_bytes(int N, int K);

int launch_forward(const HostPlan &hp, const DevicePtrs &p, void *stream);
int launch_pass1(const HostPlan &hp, const DevicePtrs &p, int g0, int ng, void *stream);
int launch_pass2(const HostPlan &hp, const DevicePtrs &p, int g0, int ng, void *stream);
int launch_finalize(const HostPlan &hp, const DevicePtrs &p, void *Q, void *Qim, void *stream);
// de-aliased plans: coefficients and f on the 2N grid before the chunks;
// projection of the 2N-grid sum onto the N_in grid after them
int launch_dealias_prepare(const HostPlan &hp, const DevicePtrs &p, void *stream);
int launch_dealias_finish(const HostPlan &hp, const DevicePtrs &p, void *Q, void *Qim, void *stream);
int launch_moments(const HostPlan &hp, const void *g, double *partials, double *out, void *stream);
int moments_partials_count(const HostPlan &hp);
int launch_rk_stage(const HostPlan &hp, const void *f, const void *k, double *kacc, void *ystage,
                    double b_s, double c_next_dt, int first, void *stream);
int launch_rk_final(const HostPlan &hp, void *f, const double *kacc, double dt, void *stream);

}  // namespace wke
