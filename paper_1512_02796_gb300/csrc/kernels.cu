// One-pass patch kernels (operator applies, diagonals, Jacobian pieces),
// the load vector, layout conversions and reductions.
#include "launch.h"

namespace qpat {

namespace {

constexpr int kRedBlocks = 608;  // 4 x 152 SMs

// ---------------------------------------------------------------- operator apply
// One CTA per patch: stage, element loop, write the owned rows.  Columns
// [c0, c0 + R) of N x ldx node-major x and y (large RHS counts are applied in
// column chunks so that the staging fits in shared memory).
template <typename T, int R, int OP>
__global__ void __launch_bounds__(kThreads) k_apply(MeshDev m, OpParams<T> op, T sign, const T* __restrict__ x,
                                                    T* __restrict__ y, int ldx, int c0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PatchSmem<T, R> s;
    s.carve(reinterpret_cast<T*>(smem_raw), m.max_touched, m.max_own);
    const int p = blockIdx.x;
    const int nb = m.node_ptr[p], nt = m.node_ptr[p + 1] - nb;
    const int ob = m.own_begin[p], nown = m.own_begin[p + 1] - ob;
    stage_static<T, R>(m, nb, nt, s, op);
    for (int i = threadIdx.x; i < nt * R; i += blockDim.x) {
        const int g = __ldg(m.nodes + nb + i / R);
        s.xin[i] = __ldg(x + size_t(g) * ldx + c0 + (i % R));
    }
    for (int i = threadIdx.x; i < nown * R; i += blockDim.x) s.yout[i] = T(0);
    __syncthreads();
    patch_elements<T, R, OP, true>(m, p, nown, s, op);  // coloured: run-to-run identical
    __syncthreads();
    for (int i = threadIdx.x; i < nown * R; i += blockDim.x) {
        T v = s.yout[i];
        if (OP == OP_PRIOR) v += op.delta * s.xin[i];
        y[size_t(ob + i / R) * ldx + c0 + (i % R)] = sign * v;
    }
}

constexpr size_t kSmemBudget = 200 * 1024;

template <typename T, int R, int OP>
cudaError_t apply_t(const MeshDev& m, const OpParams<T>& op, T sign, const T* x, T* y, int ldx, int c0,
                    cudaStream_t st) {
    const size_t smem = PatchSmem<T, R>::bytes(m.max_touched, m.max_own);
    auto kern = k_apply<T, R, OP>;
    cudaError_t e = qpat::allow_smem((const void*)kern, size_t(smem));
    if (e != cudaSuccess) return e;
    qpat::note_launch(1);
    kern<<<m.P, kThreads, smem, st>>>(m, op, sign, x, y, ldx, c0);
    return cudaGetLastError();
}

// largest chunk of {16, 8, 4, 2, 1} dividing R whose staging fits the budget
template <typename T>
int apply_chunk(const MeshDev& m, int R, size_t per_node_extra) {
    for (int c : {16, 8, 4, 2, 1}) {
        if (c > R || R % c) continue;
        const size_t bytes = sizeof(T) * (size_t(m.max_touched) * (per_node_extra + size_t(c)) +
                                          size_t(m.max_own) * c);
        if (bytes <= kSmemBudget) return c;
    }
    return 1;
}

// ---------------------------------------------------------------- diagonals (FP64)
// diag K_ii = sum_T [ S_kappa/4 |c_i|^2/(6|det|) + |T|/120 (2 S_mu + 4 mu_i) ] + sum_F |F|/12
__global__ void __launch_bounds__(kThreads) k_diag_K(MeshDev m, const double* __restrict__ kappa,
                                                     const double* __restrict__ mu, double* inv64, float* inv32) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PatchSmem<double, 1> s;
    s.carve(reinterpret_cast<double*>(smem_raw), m.max_touched, m.max_own);
    const int p = blockIdx.x;
    const int nb = m.node_ptr[p], nt = m.node_ptr[p + 1] - nb;
    const int ob = m.own_begin[p], nown = m.own_begin[p + 1] - ob;
    OpParams<double> op{kappa, mu, 0, 0, 0, 1};
    stage_static<double, 1>(m, nb, nt, s, op);
    for (int i = threadIdx.x; i < nown; i += blockDim.x) s.yout[i] = 0.0;
    __syncthreads();
    // colour by colour: plain sums in a fixed order (see for_each_coloured)
    for_each_coloured(m.tcol_beg, m.tcol_off, p, [&](int t) {
        const ushort4 lv = m.tet_loc[t];
        const int v[4] = {lv.x, lv.y, lv.z, lv.w};
        double pc[4][3], c[4][3], ad;
        load_tet(s, lv, pc);
        tet_cofactors(pc, c, ad);
        double ks = 0, Sm = 0;
        for (int a = 0; a < 4; ++a) {
            ks += s.c1[v[a]];
            Sm += s.c2[v[a]];
        }
        const double sk = ks / (24.0 * ad), vm = ad / 720.0;
        for (int a = 0; a < 4; ++a)
            if (v[a] < nown) {
                const double c2 = c[a][0] * c[a][0] + c[a][1] * c[a][1] + c[a][2] * c[a][2];
                s.yout[v[a]] += sk * c2 + vm * (2.0 * Sm + 4.0 * s.c2[v[a]]);
            }
    });
    for_each_coloured(m.fcol_beg, m.fcol_off, p, [&](int f) {
        const ushort4 lv = m.face_loc[f];
        const int v[3] = {lv.x, lv.y, lv.z};
        const double w = m.pface_area64[f] / 12.0;
        for (int a = 0; a < 3; ++a)
            if (v[a] < nown) s.yout[v[a]] += w;
    });
    for (int i = threadIdx.x; i < nown; i += blockDim.x) {
        const double d = 1.0 / s.yout[i];
        inv64[ob + i] = d;
        if (inv32) inv32[ob + i] = float(d);
    }
}

// diag M_delta: block r: scale_r c_T |c_i|^2 / (6 |det|) + delta
__global__ void __launch_bounds__(kThreads) k_diag_prior(MeshDev m, const double* __restrict__ u1,
                                                         const double* __restrict__ u2, double inv_T2,
                                                         int kind, double q, double scale1, double delta,
                                                         double* inv64, float* inv32) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PatchSmem<double, 2> s;
    s.carve(reinterpret_cast<double*>(smem_raw), m.max_touched, m.max_own);
    const int p = blockIdx.x;
    const int nb = m.node_ptr[p], nt = m.node_ptr[p + 1] - nb;
    const int ob = m.own_begin[p], nown = m.own_begin[p + 1] - ob;
    OpParams<double> op{u1, u2, inv_T2, scale1, delta, 0, nullptr, nullptr, kind, q};
    stage_static<double, 2>(m, nb, nt, s, op);
    for (int i = threadIdx.x; i < 2 * nown; i += blockDim.x) s.yout[i] = 0.0;
    __syncthreads();
    for_each_coloured(m.tcol_beg, m.tcol_off, p, [&](int t) {
        const ushort4 lv = m.tet_loc[t];
        const int v[4] = {lv.x, lv.y, lv.z, lv.w};
        double pc[4][3], c[4][3], ad;
        load_tet(s, lv, pc);
        tet_cofactors(pc, c, ad);
        for (int r = 0; r < 2; ++r) {
            const double* uc = r == 0 ? s.c1 : s.c2;
            double u[4], Gu[3];
            for (int a = 0; a < 4; ++a) u[a] = uc[v[a]];
            grad_vec(c, u, Gu);
            const double g2 = (Gu[0] * Gu[0] + Gu[1] * Gu[1] + Gu[2] * Gu[2]) / (ad * ad);
            const double cT = prior_weight<double>(kind, g2, inv_T2, q);
            const double sk = (r == 0 ? 1.0 : scale1) * cT / (6.0 * ad);
            for (int a = 0; a < 4; ++a)
                if (v[a] < nown) s.yout[2 * v[a] + r] += sk * (c[a][0] * c[a][0] + c[a][1] * c[a][1] + c[a][2] * c[a][2]);
        }
    });
    for (int i = threadIdx.x; i < 2 * nown; i += blockDim.x) {
        const double d = 1.0 / (s.yout[i] + delta);
        inv64[2 * ob + i] = d;
        if (inv32) inv32[2 * ob + i] = float(d);
    }
}

// ---------------------------------------------------------------- assembly (FP64)
// Element matrices of K (Appendix weak form) added into the owned rows of
// the sliced-ELLPACK values:  A_ab = S_kappa/(24|det|) c_a.c_b
//   + |T|/120 (a == b ? 2 S_mu + 4 mu_a : S_mu + mu_a + mu_b)   [exact P1 mass]
//   + Robin |F|/24 (1 + delta_ab) on boundary faces.
__global__ void __launch_bounds__(kThreads) k_assemble_K(MeshDev m, const double* __restrict__ kappa,
                                                         const double* __restrict__ mu, double* val) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PatchSmem<double, 1> s;
    s.carve(reinterpret_cast<double*>(smem_raw), m.max_touched, m.max_own);
    const int p = blockIdx.x;
    const int nb = m.node_ptr[p], nt = m.node_ptr[p + 1] - nb;
    const int ob = m.own_begin[p], nown = m.own_begin[p + 1] - ob;
    OpParams<double> op{kappa, mu, 0, 0, 0, 1};
    stage_static<double, 1>(m, nb, nt, s, op);
    __syncthreads();
    // colour by colour: within a colour each owned row takes one tet's terms,
    // and the barrier between colours orders the additions to an entry, so
    // the sums run in a fixed order (identical values on every run).  The
    // additions are fire-and-forget reductions into global memory (no load
    // round trip per entry); the barrier waits for them once per colour.
    for_each_coloured(m.tcol_beg, m.tcol_off, p, [&](int t) {
        const ushort4 lv = m.tet_loc[t];
        const int v[4] = {lv.x, lv.y, lv.z, lv.w};
        double pc[4][3], c[4][3], ad;
        load_tet(s, lv, pc);
        tet_cofactors(pc, c, ad);
        double ks = 0, Sm = 0;
        for (int a = 0; a < 4; ++a) {
            ks += s.c1[v[a]];
            Sm += s.c2[v[a]];
        }
        const double sk = ks / (24.0 * ad), vm = ad / 720.0;
        for (int a = 0; a < 4; ++a) {
            if (v[a] >= nown) continue;
            const int g = ob + v[a];
            for (int b = 0; b < 4; ++b) {
                const double st = sk * (c[a][0] * c[b][0] + c[a][1] * c[b][1] + c[a][2] * c[b][2]);
                const double ms = a == b ? 2.0 * Sm + 4.0 * s.c2[v[a]] : Sm + s.c2[v[a]] + s.c2[v[b]];
                const int64_t idx = sell_slot(m, g, v[b]);
                if (idx >= 0) atomicAdd(val + idx, st + vm * ms);
            }
        }
    });
    for_each_coloured(m.fcol_beg, m.fcol_off, p, [&](int f) {
        const ushort4 lv = m.face_loc[f];
        const int v[3] = {lv.x, lv.y, lv.z};
        const double w = m.pface_area64[f] / 24.0;
        for (int a = 0; a < 3; ++a) {
            if (v[a] >= nown) continue;
            for (int b = 0; b < 3; ++b) {
                const int64_t idx = sell_slot(m, ob + v[a], v[b]);
                if (idx >= 0) atomicAdd(val + idx, a == b ? 2.0 * w : w);
            }
        }
    });
}

// Prior blocks: A^r_ab = scale_r c_T(u_r) c_a.c_b / (6 |det|), c_T = r'(t)/t at t = |grad u_r| (prior_weight)
__global__ void __launch_bounds__(kThreads) k_assemble_prior(MeshDev m, const double* __restrict__ u1,
                                                             const double* __restrict__ u2, double inv_T2,
                                                             int kind, double q, double scale1, double* val0,
                                                             double* val1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PatchSmem<double, 1> s;
    s.carve(reinterpret_cast<double*>(smem_raw), m.max_touched, m.max_own);
    const int p = blockIdx.x;
    const int nb = m.node_ptr[p], nt = m.node_ptr[p + 1] - nb;
    const int ob = m.own_begin[p], nown = m.own_begin[p + 1] - ob;
    OpParams<double> op{u1, u2, 0, 0, 0, 0};
    stage_static<double, 1>(m, nb, nt, s, op);
    __syncthreads();
    // colour by colour, ordered reductions as in k_assemble_K
    for_each_coloured(m.tcol_beg, m.tcol_off, p, [&](int t) {
        const ushort4 lv = m.tet_loc[t];
        const int v[4] = {lv.x, lv.y, lv.z, lv.w};
        double pc[4][3], c[4][3], ad;
        load_tet(s, lv, pc);
        tet_cofactors(pc, c, ad);
        double coef[2];
        for (int r = 0; r < 2; ++r) {
            const double* uc = r == 0 ? s.c1 : s.c2;
            double u[4], Gu[3];
            for (int a = 0; a < 4; ++a) u[a] = uc[v[a]];
            grad_vec(c, u, Gu);
            const double g2 = (Gu[0] * Gu[0] + Gu[1] * Gu[1] + Gu[2] * Gu[2]) / (ad * ad);
            coef[r] = (r == 0 ? 1.0 : scale1) * prior_weight<double>(kind, g2, inv_T2, q) / (6.0 * ad);
        }
        for (int a = 0; a < 4; ++a) {
            if (v[a] >= nown) continue;
            const int g = ob + v[a];
            for (int b = 0; b < 4; ++b) {
                const double cc = c[a][0] * c[b][0] + c[a][1] * c[b][1] + c[a][2] * c[b][2];
                const int64_t idx = sell_slot(m, g, v[b]);
                if (idx >= 0) {
                    atomicAdd(val0 + idx, coef[0] * cc);
                    atomicAdd(val1 + idx, coef[1] * cc);
                }
            }
        }
    });
}

// val_r[diag] += shift ; inv[g * NV + r] = 1 / val_r[diag]  (FP64, optional FP32 copy).
// gbound (optional, zeroed by the caller): max over rows of sum_j |a_ij| / a_ii
// (Gershgorin: every eigenvalue of D^-1 A, and of D^-1 A_pp for a principal
// block, lies in [0, gbound] when A is symmetric positive definite).
__global__ void k_diag_csr(MeshDev m, int NV, double shift, double* val0, double* val1, double* inv64, float* inv32,
                           double* gbound) {
    double gmax = 0.0;
    for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < m.N; g += int64_t(gridDim.x) * blockDim.x) {
        const int64_t base = m.sell_ptr[g >> 5] * 32 + (g & 31);
        const int dk = m.sell_diag[g];
        const int64_t idx = base + int64_t(dk) * 32;
        for (int r = 0; r < NV; ++r) {
            double* v = r == 0 ? val0 : val1;
            const double d = v[idx] + shift;
            v[idx] = d;
            inv64[g * NV + r] = 1.0 / d;
            if (inv32) inv32[g * NV + r] = float(1.0 / d);
            if (gbound) {
                double off = 0.0;
                for (int k = 0; k < m.sell_len[g]; ++k)
                    if (k != dk) off += fabs(v[base + int64_t(k) * 32]);
                gmax = fmax(gmax, 1.0 + off / d);
            }
        }
    }
    if (gbound) {
        for (int o = 16; o > 0; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
        // non-negative doubles order like their bit patterns
        if ((threadIdx.x & 31) == 0 && gmax > 0.0)
            atomicMax(reinterpret_cast<unsigned long long*>(gbound), (unsigned long long)__double_as_longlong(gmax));
    }
}

__global__ void k_cast_vals(int64_t n, const double* in, float* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = float(in[i]);
}

// y = A x with an assembled operator: one CTA per patch, x staged on the
// touched nodes in shared memory, thread-per-row sliced-ELLPACK rows.
template <typename T, int R, int NV>
__global__ void __launch_bounds__(kThreads) k_apply_csr(MeshDev m, const T* __restrict__ v0,
                                                        const T* __restrict__ v1, const T* __restrict__ x,
                                                        T* __restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xin = reinterpret_cast<T*>(smem_raw);
    const int p = blockIdx.x;
    const int nb = m.node_ptr[p], nt = m.node_ptr[p + 1] - nb;
    const int ob = m.own_begin[p], nown = m.own_begin[p + 1] - ob;
    for (int i = threadIdx.x; i < nt * R; i += blockDim.x) {
        const int g = __ldg(m.nodes + nb + i / R);
        xin[i] = __ldg(x + size_t(g) * R + (i % R));
    }
    __syncthreads();
    csr_rows<T, R, NV>(m, ob, nown, v0, v1, xin, [&](int i, int r, T v) { y[size_t(ob + i) * R + r] = v; });
}

template <typename T, int R, int NV>
cudaError_t apply_csr_t(const MeshDev& m, const T* v0, const T* v1, const T* x, T* y, cudaStream_t st) {
    const size_t smem = sizeof(T) * size_t(m.max_touched) * R;
    auto kern = k_apply_csr<T, R, NV>;
    cudaError_t e = qpat::allow_smem((const void*)kern, size_t(smem));
    if (e != cudaSuccess) return e;
    qpat::note_launch(1);
    kern<<<m.P, kThreads, smem, st>>>(m, v0, v1, x, y);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- J^T pieces
// y[g][0] (+)= -sum_k sum_{T ni g} (|T|/4) grad(phi_k) . grad(z_k)   ( = sum_k G1^T z_k )
// y[g][1] (+)= -sum_k (M(phi_k) z_k)_g                               ( = sum_k G2 z_k )
// over the columns [c0, c0 + K) of N x ldk node-major phi and z.
template <typename T, int K>
__global__ void __launch_bounds__(kThreads) k_vjp_accum(MeshDev m, const T* __restrict__ phi,
                                                        const T* __restrict__ z, T* __restrict__ y, int ldk,
                                                        int c0, int accumulate) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int MT = m.max_touched;
    T* px = reinterpret_cast<T*>(smem_raw);
    T* py = px + MT;
    T* pz = py + MT;
    T* sphi = pz + MT;                 // MT x K
    T* sz = sphi + size_t(MT) * K;     // MT x K
    T* sy = sz + size_t(MT) * K;       // owned x 2
    const T* xyz = xyz_of<T>(m);
    const int p = blockIdx.x;
    const int nb = m.node_ptr[p], nt = m.node_ptr[p + 1] - nb;
    const int ob = m.own_begin[p], nown = m.own_begin[p + 1] - ob;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        const int g = m.nodes[nb + i];
        px[i] = xyz[3 * g];
        py[i] = xyz[3 * g + 1];
        pz[i] = xyz[3 * g + 2];
    }
    for (int i = threadIdx.x; i < nt * K; i += blockDim.x) {
        const int g = m.nodes[nb + i / K];
        sphi[i] = phi[size_t(g) * ldk + c0 + i % K];
        sz[i] = z[size_t(g) * ldk + c0 + i % K];
    }
    for (int i = threadIdx.x; i < 2 * nown; i += blockDim.x) sy[i] = T(0);
    __syncthreads();
    // colour by colour: plain sums in a fixed order (run-to-run identical)
    for_each_coloured(m.tcol_beg, m.tcol_off, p, [&](int t) {
        const ushort4 lv = m.tet_loc[t];
        const int v[4] = {lv.x, lv.y, lv.z, lv.w};
        T pc[4][3], c[4][3], ad;
        for (int a = 0; a < 4; ++a) {
            pc[a][0] = px[v[a]];
            pc[a][1] = py[v[a]];
            pc[a][2] = pz[v[a]];
        }
        tet_cofactors(pc, c, ad);
        const T s1 = T(1) / (T(24) * ad), vm = ad / T(720);
        T g1 = T(0), m4[4] = {T(0), T(0), T(0), T(0)};
        for (int k = 0; k < K; ++k) {
            T f[4], zz[4], Gf[3], Gz[3];
            for (int a = 0; a < 4; ++a) {
                f[a] = sphi[v[a] * K + k];
                zz[a] = sz[v[a] * K + k];
            }
            grad_vec(c, f, Gf);
            grad_vec(c, zz, Gz);
            g1 += Gf[0] * Gz[0] + Gf[1] * Gz[1] + Gf[2] * Gz[2];
            mass_rows_add(f, f[0] + f[1] + f[2] + f[3], zz, vm, m4);
        }
        g1 *= s1;
        for (int a = 0; a < 4; ++a)
            if (v[a] < nown) {
                sy[2 * v[a]] -= g1;
                sy[2 * v[a] + 1] -= m4[a];
            }
    });
    for (int i = threadIdx.x; i < 2 * nown; i += blockDim.x) {
        T* dst = y + size_t(ob) * 2 + i;
        *dst = accumulate ? *dst + sy[i] : sy[i];
    }
}

template <typename T, int K>
cudaError_t vjp_t(const MeshDev& m, const T* phi, const T* z, T* y, int ldk, int c0, int acc, cudaStream_t st) {
    const size_t smem = sizeof(T) * (size_t(m.max_touched) * (3 + 2 * K) + size_t(m.max_own) * 2);
    auto kern = k_vjp_accum<T, K>;
    cudaError_t e = qpat::allow_smem((const void*)kern, size_t(smem));
    if (e != cudaSuccess) return e;
    qpat::note_launch(1);
    kern<<<m.P, kThreads, smem, st>>>(m, phi, z, y, ldk, c0, acc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- load vector
// f_i += sum over the boundary faces F of node i of 2 Phi_F |F| / 3, gathered
// per (node, illumination) over the node's faces in a fixed order
__global__ void k_load(MeshDev m, int K, int R, const double* __restrict__ flux, double* f) {
    const int64_t total = int64_t(m.N) * K;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int g = int(i / K), k = int(i % K);
        const int q0 = __ldg(m.nface_ptr + g), q1 = __ldg(m.nface_ptr + g + 1);
        if (q0 == q1) continue;
        double acc = 0.0;
        for (int q = q0; q < q1; ++q) {
            const int fi = __ldg(m.nface + q);
            acc += 2.0 * __ldg(flux + size_t(k) * m.F + fi) * __ldg(m.farea + fi) / 3.0;
        }
        f[size_t(g) * R + k] += acc;
    }
}

// ---------------------------------------------------------------- layout helpers
// out[l*R + r] = in[r*N + perm[l]] for r < K, 0 for K <= r < R
template <typename Tin, typename Tout>
__global__ void k_to_lib(int N, int K, int R, const int* __restrict__ perm, const Tin* __restrict__ in,
                         Tout* __restrict__ out) {
    const int64_t total = int64_t(N) * R;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int l = int(i / R), r = int(i % R);
        out[i] = r < K ? Tout(in[int64_t(r) * N + perm[l]]) : Tout(0);
    }
}

// out[r*N + perm[l]] = in[l*R + r] for r < K
template <typename Tin, typename Tout>
__global__ void k_from_lib(int N, int K, int R, const int* __restrict__ perm, const Tin* __restrict__ in,
                           Tout* __restrict__ out) {
    const int64_t total = int64_t(N) * K;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int l = int(i / K), r = int(i % K);
        out[int64_t(r) * N + perm[l]] = Tout(in[int64_t(l) * R + r]);
    }
}

int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return int(g);
}

// ---------------------------------------------------------------- reductions
template <typename T>
__global__ void k_dot_partial(int64_t n, int R, const T* __restrict__ a, const T* __restrict__ b, double* partial) {
    // thread t handles entries i with i % R == t % R (blockDim multiple of R)
    __shared__ double sm[256];
    double acc = 0.0;
    const int64_t total = n * R;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x)
        acc += double(a[i]) * double(b[i]);
    sm[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < R) {
        double s = 0.0;
        for (int j = threadIdx.x; j < blockDim.x; j += R) s += sm[j];
        partial[size_t(blockIdx.x) * R + threadIdx.x] = s;
    }
}

__global__ void k_dot_final(int nblk, int R, const double* partial, double* out) {
    const int r = threadIdx.x;
    if (r < R) {
        double s = 0.0;
        for (int j = 0; j < nblk; ++j) s += partial[size_t(j) * R + r];
        out[r] = s;
    }
}

__global__ void k_cast_d2f_scaled(int64_t n, int R, const double* in, const double* scale, float* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n * R; i += int64_t(gridDim.x) * blockDim.x) {
        const double s = scale[i % R];
        out[i] = s > 0.0 ? float(in[i] / s) : 0.0f;
    }
}

__global__ void k_axpy_f2d_scaled(int64_t n, int R, const float* d, const double* scale, double* x) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n * R; i += int64_t(gridDim.x) * blockDim.x)
        x[i] += scale[i % R] * double(d[i]);
}

__global__ void k_sub(int64_t n, const double* a, const double* b, double* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = a[i] - b[i];
}

__global__ void k_cast_d2f(int64_t n, const double* in, float* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = float(in[i]);
}

}  // namespace

template <typename T>
cudaError_t launch_apply_K(const MeshDev& m, int R, const T* c1, const T* c2, int robin, T sign, const T* x, T* y,
                           cudaStream_t s) {
    OpParams<T> op{c1, c2, T(0), T(0), T(0), robin};
    if (R != 1 && R != 2 && R != 4 && R != 8 && R != 16) return cudaErrorInvalidValue;
    const int C = apply_chunk<T>(m, R, 5);
    for (int c0 = 0; c0 < R; c0 += C) {
        cudaError_t e = cudaErrorInvalidValue;
        switch (C) {
            case 1: e = apply_t<T, 1, OP_K>(m, op, sign, x, y, R, c0, s); break;
            case 2: e = apply_t<T, 2, OP_K>(m, op, sign, x, y, R, c0, s); break;
            case 4: e = apply_t<T, 4, OP_K>(m, op, sign, x, y, R, c0, s); break;
            case 8: e = apply_t<T, 8, OP_K>(m, op, sign, x, y, R, c0, s); break;
            case 16: e = apply_t<T, 16, OP_K>(m, op, sign, x, y, R, c0, s); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_apply_prior(const MeshDev& m, const T* u1, const T* u2, T inv_T2, int kind, T q, T scale1,
                               T delta, const T* x, T* y, cudaStream_t s) {
    OpParams<T> op{u1, u2, inv_T2, scale1, delta, 0, nullptr, nullptr, kind, q};
    return apply_t<T, 2, OP_PRIOR>(m, op, T(1), x, y, 2, 0, s);
}

cudaError_t launch_invdiag_K(const MeshDev& m, const double* kappa, const double* mu, double* inv64, float* inv32,
                             cudaStream_t s) {
    const size_t smem = PatchSmem<double, 1>::bytes(m.max_touched, m.max_own);
    cudaError_t e = qpat::allow_smem((const void*)k_diag_K, size_t(smem));
    if (e != cudaSuccess) return e;
    qpat::note_launch(1);
    k_diag_K<<<m.P, kThreads, smem, s>>>(m, kappa, mu, inv64, inv32);
    return cudaGetLastError();
}

cudaError_t launch_invdiag_prior(const MeshDev& m, const double* u1, const double* u2, double inv_T2, int kind,
                                 double q, double scale1, double delta, double* inv64, float* inv32,
                                 cudaStream_t s) {
    const size_t smem = PatchSmem<double, 2>::bytes(m.max_touched, m.max_own);
    cudaError_t e = qpat::allow_smem((const void*)k_diag_prior, size_t(smem));
    if (e != cudaSuccess) return e;
    qpat::note_launch(1);
    k_diag_prior<<<m.P, kThreads, smem, s>>>(m, u1, u2, inv_T2, kind, q, scale1, delta, inv64, inv32);
    return cudaGetLastError();
}

cudaError_t launch_assemble_K(const MeshDev& m, const double* kappa, const double* mu, double* val, double* inv64,
                              float* inv32, cudaStream_t s, double* gbound) {
    cudaError_t e = cudaMemsetAsync(val, 0, sizeof(double) * m.sell_entries, s);
    if (e != cudaSuccess) return e;
    const size_t smem = PatchSmem<double, 1>::bytes(m.max_touched, m.max_own);
    e = qpat::allow_smem((const void*)k_assemble_K, size_t(smem));
    if (e != cudaSuccess) return e;
    qpat::note_launch(1);
    k_assemble_K<<<m.P, kThreads, smem, s>>>(m, kappa, mu, val);
    if (gbound && (e = cudaMemsetAsync(gbound, 0, sizeof(double), s)) != cudaSuccess) return e;
    qpat::note_launch(1);
    k_diag_csr<<<grid_for(m.N), 256, 0, s>>>(m, 1, 0.0, val, nullptr, inv64, inv32, gbound);
    return cudaGetLastError();
}

cudaError_t launch_assemble_prior(const MeshDev& m, const double* u1, const double* u2, double inv_T2, int kind,
                                  double q, double scale1, double delta, double* val0, double* val1, double* inv64,
                                  float* inv32, cudaStream_t s, double* gbound) {
    cudaError_t e = cudaMemsetAsync(val0, 0, sizeof(double) * m.sell_entries, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(val1, 0, sizeof(double) * m.sell_entries, s);
    if (e != cudaSuccess) return e;
    const size_t smem = PatchSmem<double, 1>::bytes(m.max_touched, m.max_own);
    e = qpat::allow_smem((const void*)k_assemble_prior, size_t(smem));
    if (e != cudaSuccess) return e;
    qpat::note_launch(1);
    k_assemble_prior<<<m.P, kThreads, smem, s>>>(m, u1, u2, inv_T2, kind, q, scale1, val0, val1);
    if (gbound && (e = cudaMemsetAsync(gbound, 0, sizeof(double), s)) != cudaSuccess) return e;
    qpat::note_launch(1);
    k_diag_csr<<<grid_for(m.N), 256, 0, s>>>(m, 2, delta, val0, val1, inv64, inv32, gbound);
    return cudaGetLastError();
}

cudaError_t launch_cast_vals(int64_t n, const double* in, float* out, cudaStream_t s) {
    qpat::note_launch(1);
    k_cast_vals<<<grid_for(n), 256, 0, s>>>(n, in, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_csr(const MeshDev& m, int NV, int R, const T* v0, const T* v1, const T* x, T* y,
                             cudaStream_t s) {
    if (NV == 2) {
        if (R != 2) return cudaErrorInvalidValue;
        return apply_csr_t<T, 2, 2>(m, v0, v1, x, y, s);
    }
    switch (R) {
        case 1: return apply_csr_t<T, 1, 1>(m, v0, v1, x, y, s);
        case 2: return apply_csr_t<T, 2, 1>(m, v0, v1, x, y, s);
        case 4: return apply_csr_t<T, 4, 1>(m, v0, v1, x, y, s);
        case 8: return apply_csr_t<T, 8, 1>(m, v0, v1, x, y, s);
        case 16: return apply_csr_t<T, 16, 1>(m, v0, v1, x, y, s);
        default: return cudaErrorInvalidValue;
    }
}

// Whether k_apply_csr for R right-hand sides fits the device's per-block
// shared memory (the input vector is staged on the patch's touched nodes).
template <typename T>
bool apply_csr_fits(const MeshDev& m, int R) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return true;
    }
    return sizeof(T) * size_t(m.max_touched) * size_t(R) <= size_t(optin);
}
template bool apply_csr_fits<double>(const MeshDev&, int);
template bool apply_csr_fits<float>(const MeshDev&, int);

template cudaError_t launch_apply_csr<double>(const MeshDev&, int, int, const double*, const double*, const double*,
                                              double*, cudaStream_t);
template cudaError_t launch_apply_csr<float>(const MeshDev&, int, int, const float*, const float*, const float*,
                                             float*, cudaStream_t);

template <typename T>
cudaError_t launch_vjp_accum(const MeshDev& m, int K, const T* phi, const T* z, T* y, cudaStream_t s) {
    if (K != 1 && K != 2 && K != 4 && K != 8 && K != 16) return cudaErrorInvalidValue;
    int C = 1;
    for (int c : {16, 8, 4, 2, 1}) {
        if (c > K || K % c) continue;
        if (sizeof(T) * (size_t(m.max_touched) * (3 + 2 * c) + size_t(m.max_own) * 2) <= kSmemBudget) {
            C = c;
            break;
        }
    }
    for (int c0 = 0; c0 < K; c0 += C) {
        const int acc = c0 > 0;
        cudaError_t e = cudaErrorInvalidValue;
        switch (C) {
            case 1: e = vjp_t<T, 1>(m, phi, z, y, K, c0, acc, s); break;
            case 2: e = vjp_t<T, 2>(m, phi, z, y, K, c0, acc, s); break;
            case 4: e = vjp_t<T, 4>(m, phi, z, y, K, c0, acc, s); break;
            case 8: e = vjp_t<T, 8>(m, phi, z, y, K, c0, acc, s); break;
            case 16: e = vjp_t<T, 16>(m, phi, z, y, K, c0, acc, s); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_load(const MeshDev& m, int K, int R, const double* flux, double* f, cudaStream_t s) {
    qpat::note_launch(1);
    k_load<<<grid_for(int64_t(m.N) * K), 256, 0, s>>>(m, K, R, flux, f);
    return cudaGetLastError();
}

template <typename Tin, typename Tout>
cudaError_t launch_to_lib(const MeshDev& m, int K, int R, const Tin* in, Tout* out, cudaStream_t s) {
    qpat::note_launch(1);
    k_to_lib<Tin, Tout><<<grid_for(int64_t(m.N) * R), 256, 0, s>>>(m.N, K, R, m.perm, in, out);
    return cudaGetLastError();
}

template <typename Tin, typename Tout>
cudaError_t launch_from_lib(const MeshDev& m, int K, int R, const Tin* in, Tout* out, cudaStream_t s) {
    qpat::note_launch(1);
    k_from_lib<Tin, Tout><<<grid_for(int64_t(m.N) * K), 256, 0, s>>>(m.N, K, R, m.perm, in, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dots(int64_t n, int R, const T* a, const T* b, double* partial, double* out, cudaStream_t s) {
    qpat::note_launch(1);
    k_dot_partial<T><<<kRedBlocks, 256, 0, s>>>(n, R, a, b, partial);
    qpat::note_launch(1);
    k_dot_final<<<1, 32, 0, s>>>(kRedBlocks, R, partial, out);
    return cudaGetLastError();
}

cudaError_t launch_cast_d2f_scaled(int64_t n, int R, const double* in, const double* scale, float* out,
                                   cudaStream_t s) {
    qpat::note_launch(1);
    k_cast_d2f_scaled<<<grid_for(n * R), 256, 0, s>>>(n, R, in, scale, out);
    return cudaGetLastError();
}

cudaError_t launch_axpy_f2d_scaled(int64_t n, int R, const float* d, const double* scale, double* x,
                                   cudaStream_t s) {
    qpat::note_launch(1);
    k_axpy_f2d_scaled<<<grid_for(n * R), 256, 0, s>>>(n, R, d, scale, x);
    return cudaGetLastError();
}

cudaError_t launch_sub(int64_t n, const double* a, const double* b, double* out, cudaStream_t s) {
    qpat::note_launch(1);
    k_sub<<<grid_for(n), 256, 0, s>>>(n, a, b, out);
    return cudaGetLastError();
}

cudaError_t launch_cast_d2f(int64_t n, const double* in, float* out, cudaStream_t s) {
    qpat::note_launch(1);
    k_cast_d2f<<<grid_for(n), 256, 0, s>>>(n, in, out);
    return cudaGetLastError();
}

template cudaError_t launch_apply_K<double>(const MeshDev&, int, const double*, const double*, int, double,
                                            const double*, double*, cudaStream_t);
template cudaError_t launch_apply_K<float>(const MeshDev&, int, const float*, const float*, int, float, const float*,
                                           float*, cudaStream_t);
template cudaError_t launch_apply_prior<double>(const MeshDev&, const double*, const double*, double, int, double,
                                                double, double, const double*, double*, cudaStream_t);
template cudaError_t launch_apply_prior<float>(const MeshDev&, const float*, const float*, float, int, float, float,
                                               float, const float*, float*, cudaStream_t);
template cudaError_t launch_vjp_accum<double>(const MeshDev&, int, const double*, const double*, double*,
                                              cudaStream_t);
template cudaError_t launch_vjp_accum<float>(const MeshDev&, int, const float*, const float*, float*, cudaStream_t);
template cudaError_t launch_to_lib<double, double>(const MeshDev&, int, int, const double*, double*, cudaStream_t);
template cudaError_t launch_to_lib<double, float>(const MeshDev&, int, int, const double*, float*, cudaStream_t);
template cudaError_t launch_from_lib<double, double>(const MeshDev&, int, int, const double*, double*, cudaStream_t);
template cudaError_t launch_from_lib<float, double>(const MeshDev&, int, int, const float*, double*, cudaStream_t);
template cudaError_t launch_dots<double>(int64_t, int, const double*, const double*, double*, double*, cudaStream_t);
template cudaError_t launch_dots<float>(int64_t, int, const float*, const float*, double*, double*, cudaStream_t);

}  // namespace qpat
