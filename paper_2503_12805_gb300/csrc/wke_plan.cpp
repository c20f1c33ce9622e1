// Host side of a plan: quadrature nodes, shift vectors, field layout and
// phase tables, all in double precision (Sec. 3.3, Eq. (3.8)).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "wke_internal.h"

namespace wke {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

const char *last_error() { return g_last_error.c_str(); }

static const double kPi = 3.14159265358979323846264338327950288;

// Gauss-Legendre nodes and weights on [-1, 1], ascending, by Newton's method
// on the three-term recurrence of the Legendre polynomials.
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) {
                p1 = z;
                p0 = 1.0;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) {
                // one more evaluation of the derivative at the converged node
                double q0 = 1.0, q1 = z;
                for (int k = 2; k <= n; ++k) {
                    double q2 = ((2.0 * k - 1.0) * z * q1 - (k - 1.0) * q0) / k;
                    q0 = q1;
                    q1 = q2;
                }
                if (n == 1) {
                    q1 = z;
                    q0 = 1.0;
                }
                dp = n * (z * q1 - q0) / (z * z - 1.0);
                break;
            }
        }
        double wi = 2.0 / ((1.0 - z * z) * dp * dp);
        x[i] = -z;           // ascending order: negative roots first
        x[n - 1 - i] = z;
        w[i] = wi;
        w[n - 1 - i] = wi;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

// Sphere rules: directions (n * d) and weights (n).
static int sphere_rule(int d, int n, int rule, int param, const double *user,
                       std::vector<double> &dir, std::vector<double> &w) {
    dir.clear();
    w.clear();
    if (n < 1) return fail(WKE_ERR_INVALID, "sphere rule needs at least one point");
    if (rule == WKE_SPHERE_USER) {
        if (!user) return fail(WKE_ERR_INVALID, "WKE_SPHERE_USER needs a direction table");
        for (int i = 0; i < n; ++i) {
            double nn = 0.0;
            for (int a = 0; a < d; ++a) nn += user[i * (d + 1) + a] * user[i * (d + 1) + a];
            nn = std::sqrt(nn);
            if (!(nn > 0.0) || !std::isfinite(nn))
                return fail(WKE_ERR_INVALID, "user sphere rule has a zero or non-finite direction");
            for (int a = 0; a < d; ++a) dir.push_back(user[i * (d + 1) + a] / nn);
            w.push_back(user[i * (d + 1) + d]);
        }
        return WKE_OK;
    }
    if (d == 2) {
        if (rule != WKE_SPHERE_MIDPOINT_2D)
            return fail(WKE_ERR_INVALID, "2D supports the mid-point rule or a user rule");
        for (int p = 0; p < n; ++p) {
            double th = (p + 0.5) * 2.0 * kPi / n;
            dir.push_back(std::cos(th));
            dir.push_back(std::sin(th));
            w.push_back(2.0 * kPi / n);
        }
        return WKE_OK;
    }
    if (rule == WKE_SPHERE_PLATONIC_3D) {
        const double g = 0.5 * (1.0 + std::sqrt(5.0));   // golden ratio
        std::vector<double> v;
        auto push = [&](double x, double y, double z) {
            v.push_back(x);
            v.push_back(y);
            v.push_back(z);
        };
        auto cyc = [&](double x, double y, double z) {
            push(x, y, z);
            push(z, x, y);
            push(y, z, x);
        };
        const double s2[2] = {1.0, -1.0};
        if (n == 6) {
            for (double s : s2) push(s, 0, 0);
            for (double s : s2) push(0, s, 0);
            for (double s : s2) push(0, 0, s);
        } else if (n == 8) {
            for (double sx : s2)
                for (double sy : s2)
                    for (double sz : s2) push(sx, sy, sz);
        } else if (n == 12) {
            for (double sy : s2)
                for (double sz : s2) cyc(0.0, sy, sz * g);
        } else if (n == 20) {
            for (double sx : s2)
                for (double sy : s2)
                    for (double sz : s2) push(sx, sy, sz);
            for (double sy : s2)
                for (double sz : s2) cyc(0.0, sy / g, sz * g);
        } else {
            return fail(WKE_ERR_INVALID, "Platonic designs have 6, 8, 12 or 20 points");
        }
        for (int i = 0; i < n; ++i) {
            double nn = std::sqrt(v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] +
                                  v[3 * i + 2] * v[3 * i + 2]);
            for (int a = 0; a < 3; ++a) dir.push_back(v[3 * i + a] / nn);
            w.push_back(4.0 * kPi / n);
        }
        return WKE_OK;
    }
    if (rule == WKE_SPHERE_PRODUCT_3D) {
        int nt = param;
        if (nt < 1 || n % nt != 0)
            return fail(WKE_ERR_INVALID, "product rule: n must be a multiple of n_theta");
        int np = n / nt;
        std::vector<double> ct, wt;
        gauss_legendre(nt, ct, wt);
        for (int i = 0; i < nt; ++i) {
            double st = std::sqrt(std::max(0.0, 1.0 - ct[i] * ct[i]));
            for (int k = 0; k < np; ++k) {
                double ph = (k + 0.5) * 2.0 * kPi / np;
                dir.push_back(st * std::cos(ph));
                dir.push_back(st * std::sin(ph));
                dir.push_back(ct[i]);
                w.push_back(wt[i] * 2.0 * kPi / np);
            }
        }
        return WKE_OK;
    }
    return fail(WKE_ERR_INVALID, "unknown sphere rule");
}

// Lengths the kernels are compiled for.
static bool compiled_length(int d, int N) {
    if (d == 3) return N == 16 || N == 32 || N == 48 || N == 64;
    return N == 16 || N == 32 || N == 48 || N == 64 || N == 96 || N == 128 || N == 256;
}

// Shared-field layout: chunks of consecutive groups whose distinct fields
// stay within the product pass's limit (96 in FP32, 48 in FP64: the fields of
// a point are held in shared memory, 96 KB per block of 128 threads) and
// whose units fit the byte budget.
// Fields are the same when their shift vectors agree to 1e-12 (relative);
// the first one's shift is used.  With `force` false the layout is kept only
// when it transforms at least 15% fewer units than the per-group layout.
static int build_shared_layout(HostPlan &hp, bool force) {
    const int d = hp.d, FPG = hp.fields_per_group, PPG = hp.products_per_group;
    const int kMaxChunkFields = hp.precision == WKE_FP64 ? 48 : 96;
    size_t nd = 1;
    for (int a = 0; a < d; ++a) nd *= (size_t)hp.N;
    const size_t unit_bytes = nd * (hp.precision == WKE_FP64 ? 16 : 8);
    const size_t max_units = std::max<size_t>(1, hp.chunk_bytes / unit_bytes);

    std::vector<double> shifts;              // distinct fields of all chunks, d each
    std::vector<int> chunk_g0{0}, chunk_f0{0}, cfield(hp.n_groups);
    std::vector<int> pfa(hp.prod_fa.size()), pfb(hp.prod_fb.size());
    auto find = [&](const double *x, int f0, int f1) {
        for (int f = f0; f < f1; ++f) {
            bool same = true;
            for (int a = 0; a < d && same; ++a) {
                const double y = shifts[(size_t)f * d + a];
                same = std::fabs(y - x[a]) <= 1e-12 * (1.0 + std::fabs(x[a]));
            }
            if (same) return f;
        }
        return -1;
    };
    // local fields of group g that its C and its products use
    auto used_fields = [&](int g) {
        std::vector<int> loc{0};
        for (int p = 0; p < PPG; ++p) {
            const size_t slot = (size_t)g * PPG + p;
            if (hp.prod_W[slot] == 0.0) continue;        // padding product
            loc.push_back(hp.prod_fa[slot]);
            loc.push_back(hp.prod_fb[slot]);
        }
        return loc;
    };
    // distinct fields of groups [ga, gb)
    auto count_distinct = [&](int ga, int gb) {
        std::vector<const double *> seen;
        for (int g = ga; g < gb; ++g) {
            const double *fs = &hp.field_shift[(size_t)g * FPG * d];
            for (int l : used_fields(g)) {
                const double *x = fs + (size_t)l * d;
                bool dup = false;
                for (const double *y : seen) {
                    bool same = true;
                    for (int a = 0; a < d && same; ++a) same = std::fabs(y[a] - x[a]) <= 1e-12 * (1.0 + std::fabs(x[a]));
                    if (same) {
                        dup = true;
                        break;
                    }
                }
                if (!dup) seen.push_back(x);
            }
        }
        return (int)seen.size();
    };
    // 3D FP32 (not split): a chunk's fields must also fit the shared memory of
    // the fused axis-0 + product kernel, so that the plan can use it (at
    // N = 48 two radii of the cube rule instead of three)
    const bool fusable = d == 3 && hp.precision == WKE_FP32 && !hp.split;
    auto fits = [&](int K) {
        return K <= kMaxChunkFields && (size_t)((K + 1) / 2) <= max_units &&
               (!fusable || fused_smem_bytes(hp.N, K) <= 227 * 1024);
    };
    // Chunk boundaries: whole radial shells (the n_s groups of one radius,
    // which share most fields) while they fit; a shell too large alone is
    // split group by group.
    std::vector<int> bounds{0};
    while (bounds.back() < hp.n_groups) {
        const int start = bounds.back();
        int end = start;
        while (end < hp.n_groups) {
            const int shell_end = std::min(hp.n_groups, (end / hp.n_s + 1) * hp.n_s);
            if (!fits(count_distinct(start, shell_end))) break;
            end = shell_end;
        }
        if (end == start) {
            while (end < hp.n_groups && fits(count_distinct(start, end + 1))) ++end;
            if (end == start) end = start + 1;      // one group always forms a chunk
        }
        bounds.push_back(end);
    }
    int max_fields = 0;
    size_t next_bound = 1;
    for (int g = 0; g < hp.n_groups; ++g) {
        if (g == bounds[next_bound - 1] && g > 0) {
            chunk_g0.push_back(g);
            chunk_f0.push_back((int)(shifts.size() / d));
        }
        if (g + 1 == bounds[next_bound]) ++next_bound;
        const double *fs = &hp.field_shift[(size_t)g * FPG * d];
        const int c0 = chunk_f0.back();
        auto field_of = [&](int l) {
            const double *x = fs + (size_t)l * d;
            int f = find(x, c0, (int)(shifts.size() / d));
            if (f < 0) {
                f = (int)(shifts.size() / d);
                shifts.insert(shifts.end(), x, x + d);
            }
            return f - c0;
        };
        cfield[g] = field_of(0);
        for (int p = 0; p < PPG; ++p) {
            const size_t slot = (size_t)g * PPG + p;
            if (hp.prod_W[slot] == 0.0) {
                pfa[slot] = pfb[slot] = cfield[g];       // zero weight: any field of the chunk
                continue;
            }
            pfa[slot] = field_of(hp.prod_fa[slot]);
            pfb[slot] = field_of(hp.prod_fb[slot]);
        }
        max_fields = std::max(max_fields, (int)(shifts.size() / d) - c0);
    }
    chunk_g0.push_back(hp.n_groups);
    chunk_f0.push_back((int)(shifts.size() / d));
    const int n_chunks = (int)chunk_g0.size() - 1;

    double shared_units = 0, group_units = 0;
    for (int c = 0; c < n_chunks; ++c) shared_units += (chunk_f0[c + 1] - chunk_f0[c] + 1) / 2;
    for (int c = 0; c < hp.n_chunks; ++c) {
        const int g0 = c * hp.groups_per_chunk;
        group_units += chunk_units(hp, std::min(hp.groups_per_chunk, hp.n_groups - g0));
    }
    if (max_fields > kMaxChunkFields) {
        if (force)
            return fail(WKE_ERR_UNSUPPORTED, "shared-field layout: one group needs " + std::to_string(max_fields) +
                                                 " fields, more than the product pass holds (" +
                                                 std::to_string(kMaxChunkFields) + ")");
        return WKE_OK;
    }
    if (!force && shared_units > 0.85 * group_units) return WKE_OK;

    hp.shared = true;
    hp.field_shift = shifts;
    hp.n_fields_total = (int)(shifts.size() / d);
    hp.prod_fa = pfa;
    hp.prod_fb = pfb;
    hp.group_cfield = cfield;
    hp.chunk_g0 = chunk_g0;
    hp.chunk_f0 = chunk_f0;
    hp.n_chunks = n_chunks;
    hp.max_chunk_fields = max_fields;
    int gmax = 0;
    for (int c = 0; c < n_chunks; ++c) gmax = std::max(gmax, chunk_g0[c + 1] - chunk_g0[c]);
    hp.groups_per_chunk = gmax;
    return WKE_OK;
}

// Recognise the cube rule's structure in every chunk (HostPlan::cube).  The
// fields' shifts are classified by the signs of their components, each
// relative to the chunk's largest component (equal within 1e-9); a group
// matches when its C field is a vertex v, its three products are each one
// edge and one face field of v for distinct axes, and the three weights are
// equal.
static bool classify_cube_chunk(const HostPlan &hp, int c, HostPlan::CubeChunk &t) {
    const int g0 = hp.chunk_g0[c], g1 = hp.chunk_g0[c + 1], f0 = hp.chunk_f0[c], K = hp.chunk_f0[c + 1] - f0;
    if (g1 - g0 != 8 || K != 26) return false;
    double m = 0.0;
    for (int l = 0; l < K; ++l)
        for (int a = 0; a < 3; ++a) m = std::max(m, std::fabs(hp.field_shift[(size_t)(f0 + l) * 3 + a]));
    if (!(m > 0.0)) return false;
    std::vector<int> sg(3 * K), nz(K, 0);
    for (int l = 0; l < K; ++l)
        for (int a = 0; a < 3; ++a) {
            const double x = hp.field_shift[(size_t)(f0 + l) * 3 + a] / m;
            if (std::fabs(x) <= 1e-9) sg[3 * l + a] = 0;
            else if (std::fabs(x - 1.0) <= 1e-9) sg[3 * l + a] = 1;
            else if (std::fabs(x + 1.0) <= 1e-9) sg[3 * l + a] = -1;
            else return false;
            nz[l] += sg[3 * l + a] != 0;
        }
    std::fill(std::begin(t.edge), std::end(t.edge), -1);
    std::fill(std::begin(t.face), std::end(t.face), -1);
    std::fill(std::begin(t.cfield), std::end(t.cfield), -1);
    auto zero_axis = [&](int l) {
        for (int a = 0; a < 3; ++a)
            if (sg[3 * l + a] == 0) return a;
        return -1;
    };
    auto nonzero_axis = [&](int l) {
        for (int a = 0; a < 3; ++a)
            if (sg[3 * l + a] != 0) return a;
        return -1;
    };
    for (int l = 0; l < K; ++l) {
        if (nz[l] == 1) {
            const int i = nonzero_axis(l);
            int &e = t.edge[2 * i + (sg[3 * l + i] < 0)];
            if (e >= 0) return false;
            e = l;
        } else if (nz[l] == 2) {
            const int i = zero_axis(l), j = i == 0 ? 1 : 0, k = i == 2 ? 1 : 2;
            int &f = t.face[4 * i + (sg[3 * l + j] < 0) + 2 * (sg[3 * l + k] < 0)];
            if (f >= 0) return false;
            f = l;
        }
    }
    for (int g = g0; g < g1; ++g) {
        const int cf = hp.group_cfield[g];
        if (nz[cf] != 3) return false;
        const int v = (sg[3 * cf] < 0) + 2 * (sg[3 * cf + 1] < 0) + 4 * (sg[3 * cf + 2] < 0);
        if (t.cfield[v] >= 0) return false;
        t.cfield[v] = cf;
        t.w[v] = hp.prod_W[(size_t)g * 3];
        int axes = 0;
        for (int q = 0; q < 3; ++q) {
            const size_t slot = (size_t)g * 3 + q;
            if (hp.prod_W[slot] != t.w[v]) return false;
            int fe = hp.prod_fa[slot], ff = hp.prod_fb[slot];
            if (nz[fe] == 2) std::swap(fe, ff);
            if (nz[fe] != 1 || nz[ff] != 2) return false;
            const int i = nonzero_axis(fe);
            if (zero_axis(ff) != i || (axes >> i) & 1) return false;
            axes |= 1 << i;
            for (int a = 0; a < 3; ++a)
                if ((a == i ? sg[3 * fe + a] : sg[3 * ff + a]) != sg[3 * cf + a]) return false;
        }
    }
    for (int i = 0; i < 6; ++i)
        if (t.edge[i] < 0) return false;
    for (int i = 0; i < 12; ++i)
        if (t.face[i] < 0) return false;
    for (int i = 0; i < 8; ++i)
        if (t.cfield[i] < 0) return false;
    return true;
}

static void build_cube_schedule(HostPlan &hp) {
    hp.cube.clear();
    if (!(hp.shared && hp.d == 3 && hp.N == 64 && hp.products_per_group == 3)) return;   // k_fused64's schedule
    std::vector<HostPlan::CubeChunk> tabs(hp.n_chunks);
    for (int c = 0; c < hp.n_chunks; ++c)
        if (!classify_cube_chunk(hp, c, tabs[c])) return;
    hp.cube = tabs;
}

// Order the fields of every chunk of the cube rule's form as the fused
// kernel reads them: the edge fields (index 2 i + [sign < 0]), then the face
// fields (index 4 i + q), then the C fields by vertex, so that the two
// fields of each unit (fields 2u, 2u + 1) are read together in the product
// phase: edges +-e_i, two faces of the same axis, the C fields of two
// vertices.  A renaming of the chunk's field ids (shifts, products and C
// fields follow it); the evaluation is the same up to rounding.
static void order_cube_fields(HostPlan &hp) {
    if (!(hp.shared && hp.d == 3 && hp.N == 64 && hp.products_per_group == 3)) return;
    std::vector<HostPlan::CubeChunk> tabs(hp.n_chunks);
    for (int c = 0; c < hp.n_chunks; ++c)
        if (!classify_cube_chunk(hp, c, tabs[c])) return;
    for (int c = 0; c < hp.n_chunks; ++c) {
        const HostPlan::CubeChunk &t = tabs[c];
        const int f0 = hp.chunk_f0[c];
        int perm[26];    // old chunk-local id -> new
        for (int k = 0; k < 6; ++k) perm[t.edge[k]] = k;
        for (int k = 0; k < 12; ++k) perm[t.face[k]] = 6 + k;
        for (int v = 0; v < 8; ++v) perm[t.cfield[v]] = 18 + v;
        std::vector<double> sh(hp.field_shift.begin() + (size_t)f0 * 3, hp.field_shift.begin() + (size_t)(f0 + 26) * 3);
        for (int l = 0; l < 26; ++l)
            for (int a = 0; a < 3; ++a) hp.field_shift[(size_t)(f0 + perm[l]) * 3 + a] = sh[(size_t)l * 3 + a];
        for (int g = hp.chunk_g0[c]; g < hp.chunk_g0[c + 1]; ++g) {
            hp.group_cfield[g] = perm[hp.group_cfield[g]];
            for (int q = 0; q < 3; ++q) {
                const size_t slot = (size_t)g * 3 + q;
                hp.prod_fa[slot] = perm[hp.prod_fa[slot]];
                hp.prod_fb[slot] = perm[hp.prod_fb[slot]];
            }
        }
    }
}

// Separable transforms (3D, shared-field layout; see HostPlan::separable).
// Row values and pairs are equal when they agree to 1e-12 (relative), as
// fields are; the first field with a value supplies its phase row.  With
// `force` false the layout is kept when the row-value and pair transforms
// are at most 85% of the two trailing-axis transforms of every unit.
static int build_separable(HostPlan &hp, bool force) {
    const int d = hp.d;
    std::vector<int> chunk_v0{0}, chunk_p0{0}, sep_v, sep_p, field_pair(hp.n_fields_total, 0);
    double sep_cost = 0.0, unit_cost = 0.0;
    int maxp = 0, maxv = 0;
    auto same = [](double a, double b) { return std::fabs(a - b) <= 1e-12 * (1.0 + std::fabs(a)); };
    for (int c = 0; c < hp.n_chunks; ++c) {
        const int f0 = hp.chunk_f0[c], f1 = hp.chunk_f0[c + 1];
        std::vector<int> vrep;                     // field of each row value
        std::vector<std::vector<int>> prep;        // per row value: field of each pair
        std::vector<int> fv(f1 - f0), fp(f1 - f0);
        for (int f = f0; f < f1; ++f) {
            const double *x = &hp.field_shift[(size_t)f * d];
            int vi = -1;
            for (size_t k = 0; k < vrep.size() && vi < 0; ++k)
                if (same(hp.field_shift[(size_t)vrep[k] * d + 2], x[2])) vi = (int)k;
            if (vi < 0) {
                vi = (int)vrep.size();
                vrep.push_back(f);
                prep.emplace_back();
            }
            int pi = -1;
            for (size_t k = 0; k < prep[vi].size() && pi < 0; ++k)
                if (same(hp.field_shift[(size_t)prep[vi][k] * d + 1], x[1])) pi = (int)k;
            if (pi < 0) {
                pi = (int)prep[vi].size();
                prep[vi].push_back(f);
            }
            fv[f - f0] = vi;
            fp[f - f0] = pi;
        }
        std::vector<int> first(vrep.size() + 1, 0);
        for (size_t k = 0; k < vrep.size(); ++k) first[k + 1] = first[k] + (int)prep[k].size();
        for (size_t k = 0; k < vrep.size(); ++k) {
            sep_v.push_back(vrep[k]);
            sep_v.push_back(first[k]);
            sep_v.push_back(first[k + 1]);
            for (int pf : prep[k]) sep_p.push_back(pf);
        }
        for (int f = f0; f < f1; ++f) field_pair[f] = first[fv[f - f0]] + fp[f - f0];
        chunk_v0.push_back((int)(sep_v.size() / 3));
        chunk_p0.push_back((int)sep_p.size());
        maxv = std::max(maxv, (int)vrep.size());
        maxp = std::max(maxp, first.back());
        sep_cost += (double)vrep.size() + first.back();
        unit_cost += 2.0 * ((f1 - f0 + 1) / 2);
    }
    if (!force && sep_cost > 0.85 * unit_cost) return WKE_OK;
    hp.separable = true;
    hp.chunk_v0 = chunk_v0;
    hp.chunk_p0 = chunk_p0;
    hp.sep_v = sep_v;
    hp.sep_p = sep_p;
    hp.field_pair = field_pair;
    hp.max_chunk_pairs = maxp;
    hp.max_chunk_values = maxv;
    return WKE_OK;
}

// Product-pass limits of the fused axis-0 + product kernel: the chunk's
// product table travels as a kernel parameter.
constexpr int kFusedMaxProducts = 256, kFusedMaxGroups = 64;

// Dynamic shared memory of the fused kernel for a 3D FP32 transform grid N
// and K fields: twiddles, K field slots of the block's N * LPW points and a
// padded exchange line for each line of each warp (LineCfg / LinePad of the
// kernels: 8 points per thread, 12 for N = 48).
size_t fused_smem_bytes(int N, int K) {
    const int E = N % 3 == 0 ? 12 : 8, TPL = N / E, LPW = 32 / TPL;
    const int len = N + N / 8, pitch = len + ((4 - (len % 16)) + 16) % 16;
    const int pts = N * LPW, warps = pts / 32;
    return (size_t)(N + (size_t)K * pts + (size_t)warps * LPW * pitch) * 8;
}

int build_host_plan(int d, int N, double L, int M, const wke_quadrature *quad, HostPlan &hp) {
    if (!quad) return fail(WKE_ERR_INVALID, "quadrature descriptor is NULL");
    if (d != 2 && d != 3) return fail(WKE_ERR_INVALID, "d must be 2 or 3");
    if (!(L > 0.0) || !std::isfinite(L)) return fail(WKE_ERR_INVALID, "L must be positive");
    if (N < 2 || N % 2) return fail(WKE_ERR_INVALID, "N must be even and >= 2");
    if (quad->n_r < 1 || quad->n_s < 1 || quad->n_sig < 1)
        return fail(WKE_ERR_INVALID, "n_r, n_s and n_sig must be >= 1");
    if ((long long)quad->n_r * quad->n_s * quad->n_sig != (long long)M)
        return fail(WKE_ERR_INVALID, "M must equal n_r * n_s * n_sig");
    if (quad->precision != WKE_FP64 && quad->precision != WKE_FP32 && quad->precision != WKE_SPLIT)
        return fail(WKE_ERR_INVALID, "precision must be WKE_FP64, WKE_FP32 or WKE_SPLIT");
    if (quad->precision == WKE_SPLIT && quad->layout == WKE_LAYOUT_PER_GROUP)
        return fail(WKE_ERR_INVALID, "WKE_SPLIT needs the shared-field layout");
    if (quad->nyquist != WKE_NYQ_KEEP && quad->nyquist != WKE_NYQ_ZERO)
        return fail(WKE_ERR_INVALID, "nyquist must be WKE_NYQ_KEEP or WKE_NYQ_ZERO");
    if (quad->dispersion != WKE_OMEGA_HALF_K2 && quad->dispersion != WKE_OMEGA_K2)
        return fail(WKE_ERR_INVALID, "unknown dispersion");
    if (!(quad->R >= 0.0) || !std::isfinite(quad->R)) return fail(WKE_ERR_INVALID, "R must be >= 0");
    if (quad->alias != WKE_ALIAS_CIRCULAR && quad->alias != WKE_DEALIAS_PAD2)
        return fail(WKE_ERR_INVALID, "alias must be WKE_ALIAS_CIRCULAR or WKE_DEALIAS_PAD2");
    const bool dealias = quad->alias == WKE_DEALIAS_PAD2;
    if (dealias && quad->nyquist != WKE_NYQ_ZERO)
        return fail(WKE_ERR_INVALID, "WKE_DEALIAS_PAD2 needs WKE_NYQ_ZERO: a kept -N/2 mode has no partner on "
                                     "the 2N grid, so the padded fields would not be real");
    if (!compiled_length(d, N) || !compiled_length(d, dealias ? 2 * N : N))
        return fail(WKE_ERR_UNSUPPORTED,
                    "kernels are built for N in {16, 32, 48, 64, 96, 128, 256} (2D) or {16, 32, 48, 64} (3D); "
                    "a de-aliased plan also needs 2N in that set");

    hp = HostPlan();
    hp.d = d;
    hp.N = dealias ? 2 * N : N;
    hp.N_in = N;
    hp.dealias = dealias;
    hp.M = M;
    hp.L = L;
    hp.R = quad->R > 0.0 ? quad->R : 4.0 * L / (3.0 + std::sqrt(2.0));
    hp.n_r = quad->n_r;
    hp.n_s = quad->n_s;
    hp.n_sig = quad->n_sig;
    hp.split = quad->precision == WKE_SPLIT;
    hp.precision = hp.split ? WKE_FP32 : quad->precision;
    hp.nyquist = quad->nyquist;
    hp.dispersion = quad->dispersion;

    // Radial rule: Gauss-Legendre mapped to [0, R].
    std::vector<double> x, wx;
    gauss_legendre(hp.n_r, x, wx);
    for (int i = 0; i < hp.n_r; ++i) {
        hp.r.push_back(0.5 * hp.R * (x[i] + 1.0));
        hp.w_r.push_back(0.5 * hp.R * wx[i]);
    }
    int rule_s = quad->sphere_rule < 0 ? (d == 2 ? WKE_SPHERE_MIDPOINT_2D : WKE_SPHERE_PLATONIC_3D)
                                       : quad->sphere_rule;
    int rule_g = quad->sphere_rule_sig < 0 ? rule_s : quad->sphere_rule_sig;
    int param_g = quad->sphere_rule_sig < 0 ? quad->sphere_param : quad->sphere_param_sig;
    int rc = sphere_rule(d, hp.n_s, rule_s, quad->sphere_param, quad->user_s, hp.qhat, hp.w_s);
    if (rc) return rc;
    rc = sphere_rule(d, hp.n_sig, rule_g, param_g,
                     quad->sphere_rule_sig < 0 && rule_g == WKE_SPHERE_USER ? quad->user_s
                                                                           : quad->user_sig,
                     hp.sig, hp.w_sig);
    if (rc) return rc;

    // Antipodal pairing of the sigma rule: sigma_{p'} = -sigma_p with equal
    // weights makes f_N(k - b_p) identical to f_N(k - a_{p'}) and the node
    // products of p and p' identical.
    hp.paired = false;
    if (quad->pair_antipodal && hp.n_sig % 2 == 0) {
        hp.anti.assign(hp.n_sig, -1);
        bool ok = true;
        for (int i = 0; i < hp.n_sig && ok; ++i) {
            int found = -1;
            for (int k = 0; k < hp.n_sig; ++k) {
                if (k == i) continue;
                double dev = 0.0;
                for (int a = 0; a < d; ++a) dev = std::max(dev, std::fabs(hp.sig[k * d + a] + hp.sig[i * d + a]));
                if (dev < 1e-13 && std::fabs(hp.w_sig[k] - hp.w_sig[i]) <= 1e-14 * std::fabs(hp.w_sig[i])) {
                    found = k;
                    break;
                }
            }
            if (found < 0) ok = false;
            hp.anti[i] = found;
        }
        if (ok) {
            hp.paired = true;
            // make the pairs exactly antipodal so the shared fields coincide
            for (int i = 0; i < hp.n_sig; ++i)
                if (hp.anti[i] > i)
                    for (int a = 0; a < d; ++a) hp.sig[hp.anti[i] * d + a] = -hp.sig[i * d + a];
        } else {
            hp.anti.clear();
        }
    }

    // Nodes in (p1, p2, p3) order.
    hp.W.resize(M);
    hp.q.resize((size_t)M * d);
    hp.a.resize((size_t)M * d);
    hp.b.resize((size_t)M * d);
    int p = 0;
    for (int p1 = 0; p1 < hp.n_r; ++p1) {
        double r = hp.r[p1];
        double rw = hp.w_r[p1] * std::pow(r, 2 * d - 3);
        for (int p2 = 0; p2 < hp.n_s; ++p2) {
            for (int p3 = 0; p3 < hp.n_sig; ++p3, ++p) {
                hp.W[p] = rw * hp.w_s[p2] * hp.w_sig[p3];
                for (int a = 0; a < d; ++a) {
                    double qa = r * hp.qhat[p2 * d + a];
                    double sa = r * hp.sig[p3 * d + a];
                    hp.q[(size_t)p * d + a] = qa;
                    hp.a[(size_t)p * d + a] = 0.5 * (qa - sa);
                    hp.b[(size_t)p * d + a] = 0.5 * (qa + sa);
                }
            }
        }
    }

    // Field and product layout per group.  With pairing, local field 1 + i
    // is f_N(k - a_i); the product of the pair (i, anti(i)) takes fields
    // 1 + i and 1 + anti(i).  Without it, fields 1 + 2i and 2 + 2i are A_i and B_i.
    hp.n_groups = hp.n_r * hp.n_s;
    std::vector<int> base_fa, base_fb, base_node;     // base products: local fields, first sigma index
    if (hp.paired) {
        hp.fields_per_group = 1 + hp.n_sig;
        for (int i = 0; i < hp.n_sig; ++i)
            if (hp.anti[i] > i) {
                base_fa.push_back(1 + i);
                base_fb.push_back(1 + hp.anti[i]);
                base_node.push_back(i);
            }
    } else {
        hp.fields_per_group = 1 + 2 * hp.n_sig;
        for (int i = 0; i < hp.n_sig; ++i) {
            base_fa.push_back(1 + 2 * i);
            base_fb.push_back(2 + 2 * i);
            base_node.push_back(i);
        }
    }
    // Vanishing nodes.  For sigma = qhat, k' = k and k2' = k - q (a = 0,
    // b = q); for sigma = -qhat the two swap.  Then A = F and B = C (or the
    // reverse) and A B (C + F) - C F (A + B) = 0 identically, provided F is
    // the interpolant's value f_N(k): true on the grid when the Nyquist modes
    // are kept, and on the 2N grid of a de-aliased plan; not with the modes
    // zeroed on the N grid, where F = f(k) differs from f_N(k).  With pairing
    // on, such products are dropped (an exact simplification, like the
    // pairing); without it every node is evaluated as Algorithm 1 loops.
    const bool drop = hp.paired && (hp.nyquist == WKE_NYQ_KEEP || hp.dealias);
    std::vector<std::vector<int>> keep(hp.n_groups);
    size_t ppg = 0;
    for (int g = 0; g < hp.n_groups; ++g) {
        const int p2 = g % hp.n_s;
        for (size_t k = 0; k < base_fa.size(); ++k) {
            const int i = base_node[k];
            double dp = 0.0, dm = 0.0;
            for (int a = 0; a < d; ++a) {
                dp = std::max(dp, std::fabs(hp.sig[i * d + a] - hp.qhat[p2 * d + a]));
                dm = std::max(dm, std::fabs(hp.sig[i * d + a] + hp.qhat[p2 * d + a]));
            }
            if (!(drop && (dp < 1e-13 || dm < 1e-13))) keep[g].push_back((int)k);
        }
        ppg = std::max(ppg, keep[g].size());
    }
    // a uniform count per group (groups with fewer get zero-weight padding)
    hp.products_per_group = (int)std::max<size_t>(1, ppg);
    hp.field_shift.assign((size_t)hp.n_groups * hp.fields_per_group * d, 0.0);
    hp.prod_W.assign((size_t)hp.n_groups * hp.products_per_group, 0.0);
    hp.prod_fa.assign((size_t)hp.n_groups * hp.products_per_group, base_fa[0]);
    hp.prod_fb.assign((size_t)hp.n_groups * hp.products_per_group, base_fb[0]);
    for (int g = 0; g < hp.n_groups; ++g) {
        int node0 = g * hp.n_sig;
        double *fs = &hp.field_shift[(size_t)g * hp.fields_per_group * d];
        for (int a = 0; a < d; ++a) fs[a] = hp.q[(size_t)node0 * d + a];
        for (int i = 0; i < hp.n_sig; ++i) {
            int node = node0 + i;
            if (hp.paired) {
                for (int a = 0; a < d; ++a) fs[(1 + i) * d + a] = hp.a[(size_t)node * d + a];
            } else {
                for (int a = 0; a < d; ++a) {
                    fs[(1 + 2 * i) * d + a] = hp.a[(size_t)node * d + a];
                    fs[(2 + 2 * i) * d + a] = hp.b[(size_t)node * d + a];
                }
            }
        }
        for (size_t j = 0; j < keep[g].size(); ++j) {
            const int k = keep[g][j], i = base_node[k];
            const size_t slot = (size_t)g * hp.products_per_group + j;
            hp.prod_fa[slot] = base_fa[k];
            hp.prod_fb[slot] = base_fb[k];
            hp.prod_W[slot] = hp.paired ? hp.W[node0 + i] + hp.W[node0 + hp.anti[i]] : hp.W[node0 + i];
        }
    }

    // Chunks of groups whose intermediate fields fit the byte budget.
    size_t cxb = hp.precision == WKE_FP64 ? 16 : 8;
    size_t nd = 1;
    for (int a = 0; a < d; ++a) nd *= (size_t)hp.N;
    // two groups share one C unit, so a group costs products + 1/2 units
    size_t per_pair = (size_t)(2 * hp.products_per_group + 1) * nd * cxb;
    // default budget: 48 MiB in FP32 (a 3D N=64 radius of 13 units, 27 MB, double-buffered in
    // L2); 64 MiB in FP64, whose ALU-bound passes gain more from keeping a radius whole (54 MB)
    // than from L2 residency
    hp.chunk_bytes = quad->chunk_bytes ? quad->chunk_bytes : (size_t)(hp.precision == WKE_FP64 ? 64 : 48) << 20;
    hp.groups_per_chunk = (int)std::max<size_t>(1, 2 * (hp.chunk_bytes / per_pair));
    hp.groups_per_chunk = std::min(hp.groups_per_chunk, hp.n_groups);
    hp.n_chunks = (hp.n_groups + hp.groups_per_chunk - 1) / hp.groups_per_chunk;
    hp.n_fields_total = hp.n_groups * hp.fields_per_group;

    if (quad->layout != WKE_LAYOUT_AUTO && quad->layout != WKE_LAYOUT_PER_GROUP && quad->layout != WKE_LAYOUT_SHARED &&
        quad->layout != WKE_LAYOUT_SEPARABLE)
        return fail(WKE_ERR_INVALID, "layout must be WKE_LAYOUT_AUTO, _PER_GROUP, _SHARED or _SEPARABLE");
    if (quad->layout == WKE_LAYOUT_SEPARABLE && (d != 3 || hp.split))
        return fail(WKE_ERR_INVALID, "WKE_LAYOUT_SEPARABLE needs d = 3 and is not available with WKE_SPLIT");
    if (quad->layout != WKE_LAYOUT_PER_GROUP) {
        int rc2 = build_shared_layout(hp, quad->layout == WKE_LAYOUT_SHARED || quad->layout == WKE_LAYOUT_SEPARABLE ||
                                              hp.split);
        if (rc2) return rc2;
    }
    if (hp.split && (d != 3 || (hp.N != 32 && hp.N != 64)))
        return fail(WKE_ERR_UNSUPPORTED, "WKE_SPLIT is built for 3D transform grids of N = 32 or 64");
    if (hp.shared && d == 3 && hp.precision == WKE_FP32 && !hp.split) order_cube_fields(hp);
    if (hp.shared && d == 3 && !hp.split && quad->layout != WKE_LAYOUT_SHARED) {
        int rc2 = build_separable(hp, quad->layout == WKE_LAYOUT_SEPARABLE);
        if (rc2) return rc2;
    }
    if (hp.shared && d == 3 && hp.precision == WKE_FP32 && !hp.split) {
        int maxp = 0;
        for (int c = 0; c < hp.n_chunks; ++c)
            maxp = std::max(maxp, (hp.chunk_g0[c + 1] - hp.chunk_g0[c]) * hp.products_per_group);
        hp.can_fuse = hp.groups_per_chunk <= kFusedMaxGroups && maxp <= kFusedMaxProducts &&
                      hp.max_chunk_fields <= 255 && fused_smem_bytes(hp.N, hp.max_chunk_fields) <= 227 * 1024;
        hp.fused = hp.can_fuse;
        if (hp.can_fuse) build_cube_schedule(hp);
    }
    if (hp.shared) {
        hp.chunk_u0.assign(1, 0);
        for (int c = 0; c < hp.n_chunks; ++c) hp.chunk_u0.push_back(hp.chunk_u0.back() + units_of_chunk(hp, c));
    }

    hp.scale = std::ldexp(1.0, 1 - d) * (hp.dispersion == WKE_OMEGA_K2 ? 0.5 : 1.0);
    return WKE_OK;
}

void phase_row(int N, double L, double x, double *out) {
    for (int pos = 0; pos < N; ++pos) {
        int j = pos < N / 2 ? pos : pos - N;      // signed mode, -N/2 at pos N/2
        double th = -kPi * (double)j * x / L;
        out[2 * pos] = std::cos(th);
        out[2 * pos + 1] = std::sin(th);
    }
}

static size_t grid_size(const HostPlan &hp);

size_t chunk_unit_bytes(const HostPlan &hp) {
    size_t cxb = hp.precision == WKE_FP64 ? 16 : 8;
    return std::max((size_t)max_chunk_units(hp) * grid_size(hp) * cxb, grid_size(hp) * 16);
}

size_t chunk_v_bytes(const HostPlan &hp) {
    size_t cxb = hp.precision == WKE_FP64 ? 16 : 8;   // a unit's two fields interleaved
    return (size_t)max_chunk_units(hp) * hp.d * (grid_size(hp) / hp.N) * cxb;
}

size_t chunk_s_bytes(const HostPlan &hp) {
    size_t cxb = hp.precision == WKE_FP64 ? 16 : 8;
    return (size_t)hp.max_chunk_pairs * grid_size(hp) * cxb;
}

// Kernels one evaluation launches: the forward transform (d line kernels),
// per chunk the Nyquist tables (Nyquist kept), the trailing-axis pass, the
// axis-0 transform (shared layout, unless fused with the products) and the
// product pass, then finalize (de-aliased plans: 1 padding + d maps before,
// 1 + d maps after instead of finalize; fused plans write Q in the last
// chunk's product kernel instead).
int launches_per_collision(const HostPlan &hp) {
    int per_chunk = (hp.nyquist == WKE_NYQ_KEEP ? 1 : 0) + 2 + (hp.shared && !hp.fused ? 1 : 0);
    int n = hp.d + per_chunk * hp.n_chunks + (hp.fused && !hp.dealias ? 0 : 1);
    if (hp.dealias) n += 1 + hp.d + hp.d;
    return n;
}

static size_t grid_size(const HostPlan &hp) {
    size_t nd = 1;
    for (int a = 0; a < hp.d; ++a) nd *= (size_t)hp.N;
    return nd;
}

size_t plan_device_bytes(const HostPlan &hp) {
    size_t nd = grid_size(hp);
    size_t tb = hp.precision == WKE_FP64 ? 8 : 4;
    size_t cxb = 2 * tb;
    size_t n_fields = (size_t)hp.n_fields_total;
    size_t bytes = 0;
    bytes += nd * cxb + hp.d * (nd / hp.N) * cxb;                       // ghat, Nyquist slices
    if (needs_unit_buffers(hp)) bytes += 2 * chunk_unit_bytes(hp);     // H double-buffered
    if (hp.separable) bytes += 2 * std::max(chunk_s_bytes(hp), nd * 16); // S double-buffered (S[0] also
                                                                        // the forward scratch)
    if (hp.separable)
        bytes += (hp.sep_v.size() + hp.sep_p.size() + hp.field_pair.size()) * sizeof(int);
    if (hp.separable && hp.can_fuse) bytes += (size_t)total_units(hp) * hp.N * 16;   // unit axis-0 phases
    if (hp.nyquist == WKE_NYQ_KEEP) bytes += 2 * chunk_v_bytes(hp);      // Nyquist tables, double-buffered
    bytes += 2 * (size_t)(hp.shared ? 1 : hp.groups_per_chunk) * nd * 8;   // Qacc, Qacc_im
    bytes += (size_t)hp.n_groups * sizeof(int);                         // C field of each group
    bytes += n_fields * hp.d * hp.N * cxb;                              // phase tables
    bytes += hp.N * cxb + hp.N * 16;                                    // twiddles
    bytes += (size_t)hp.n_groups * hp.products_per_group * 2 * sizeof(int);
    bytes += (size_t)hp.n_groups * hp.products_per_group * 8;
    size_t nin = 1;
    for (int a = 0; a < hp.d; ++a) nin *= (size_t)hp.N_in;
    bytes += 2 * nin * tb;                                              // host-call staging
    bytes += 2 * nin * tb + nin * 8;                                    // RK stage, k, k-sum
    if (hp.dealias)                                                     // f and Q on the 2N grid,
        bytes += nd * tb + 2 * nd * 16 + nin * cxb                      // two map buffers, coarse ghat,
                 + 2 * (size_t)hp.N * hp.N_in * 16;                     // interpolation / projection
    bytes += (size_t)moments_partials_count(hp) * (hp.d + 2) * 8 + (hp.d + 2) * 8;
    return bytes;
}

// Units transformed per evaluation.
double total_units(const HostPlan &hp) {
    double u = 0;
    for (int c = 0; c < hp.n_chunks; ++c) u += units_of_chunk(hp, c);
    return u;
}

double plan_flops(const HostPlan &hp) {
    double nd = (double)grid_size(hp);
    double lg = std::log2(nd);
    double units = total_units(hp);
    double n_fields = 2.0 * units;
    double n_prod = (double)hp.n_groups * hp.products_per_group;
    double nin = std::pow((double)hp.N_in, hp.d);
    double fwd = 5.0 * nin * std::log2(nin);
    if (hp.dealias) {                                      // per-axis interpolation and projection maps
        double maps = 0, size = nin;
        for (int a = 0; a < hp.d; ++a) { size = size / hp.N_in * hp.N; maps += size * hp.N_in * 8.0; }
        size = nd;
        for (int a = 0; a < hp.d; ++a) { size = size / hp.N * hp.N_in; maps += size * hp.N * 8.0; }
        fwd += maps;
    }
    double inv = units * 5.0 * nd * lg;                    // pass 1 + pass 2 transforms
    if (hp.separable) {
        // trailing axes once per row value (axis 2) and once per pair (axis 1),
        // axis 0 per unit
        double vals = (double)(hp.chunk_v0.back()), pairs = (double)(hp.chunk_p0.back());
        inv = (vals + pairs) * 5.0 * nd * std::log2((double)hp.N) + units * 5.0 * nd * std::log2((double)hp.N);
    }
    // per-group layout: pass 2 transforms each group's C unit once per group
    double c_again = hp.shared ? 0.0
                               : ((double)hp.n_groups - (units - n_prod)) * 5.0 * nd * std::log2((double)hp.N);
    (void)n_fields;
    // Nyquist tables: d transforms of N^{d-1} points per unit (two fields each)
    double nyq = hp.nyquist == WKE_NYQ_KEEP ? units * hp.d * 5.0 * (nd / hp.N) * std::log2(nd / hp.N) : 0.0;
    double phases = units * nd * 16.0;                     // two phase products and the packing per point
    if (hp.separable)                                      // a phase product per row value and pair, two per unit
        phases = (double)(hp.chunk_v0.back() + hp.chunk_p0.back()) * nd * 6.0 + units * nd * 14.0;
    double prods = n_prod * nd * 30.0;                     // cubic product, weight, accumulate
    return fwd + inv + c_again + nyq + phases + prods;
}

double plan_l2_bytes(const HostPlan &hp) {
    double nd = (double)grid_size(hp);
    double cxb = hp.precision == WKE_FP64 ? 16.0 : 8.0;
    return total_units(hp) * nd * cxb * 2.0;  // each unit written once, read (about) once
}

}  // namespace wke
