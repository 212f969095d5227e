// Solve kernels: one CTA per partition, double-float arithmetic; the
// per-partition work of solve_init and solve_iter is in mf_solve_body.cuh.
// solve_literal (literal schedule, Fig. 1 as printed): assemble C^k from a
//   fresh statistics pass over d_i, factorise and solve, every iteration.
#include "mf_solve_body.cuh"

namespace mf {

size_t solve_init_smem_bytes(int B, int BA) {
  const int K = BA - B;  // at most the directions + 2 of the augmented width (upper bound)
  return ((size_t)BA * BA + (8 + K + 2) * (size_t)B) * sizeof(df) + (size_t)K * B * sizeof(float) +
         64;
}
size_t solve_iter_smem_bytes(int B) {
  return ((size_t)B * linv_ld(B) + 16 * (size_t)B + 8) * sizeof(df) + 64;
}
size_t solve_literal_smem_bytes(int B, int BA) {
  const int K = BA - B;
  return ((size_t)BA * BA + (6 + K + 2) * (size_t)B) * sizeof(df) + (size_t)K * B * sizeof(float) +
         64;
}

__global__ void __launch_bounds__(kThreads, 4) solve_init_kernel(Params p) {
  prefetch_pixel_pass(p, 0);  // the cube only: no need to wait
  pdl_wait();
  pdl_trigger();
  const LaunchSpan span(p);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  solve_init_part<false>(p, blockIdx.x, smem_raw);
}

__global__ void __launch_bounds__(kThreads, 4) solve_iter_kernel(Params p, int mode, int pass) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t s_xbar;
  uint32_t ph_x = 0;
  solve_iter_part<false>(p, mode, pass, blockIdx.x, smem_raw, &s_xbar, ph_x, [] { return true; });
}

__global__ void __launch_bounds__(kThreads, 4) solve_literal_kernel(Params p, int pass) {
  pdl_wait();
  pdl_trigger();
  const LaunchSpan span(p);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ df red[kWarps];
  const int part = blockIdx.x;
  const int tid = threadIdx.x;
  const int B = p.B, BA = p.BA, K = p.K;
  const size_t pb = (size_t)part * B;
  if (p.status[part] != MF_OK) return;
  if (pass > p.lines[part_line(p, part)].n_iter) return;  // the line's iterations are done
  const DfMat A{reinterpret_cast<float*>(smem_raw), BA, BA * BA};
  df* u1 = reinterpret_cast<df*>(smem_raw) + (size_t)BA * BA;  // mu0f
  df* u2 = u1 + B;               // t^k
  df* u3 = u2 + B;               // sum c_k q_k - mu^k
  df* vz = u3 + B;
  df* invd = vz + B;
  df* vd = invd + B;             // mu^k - mu0f
  df* scr = vd + B;              // (K + 2) B: assemble's scratch, later the solve's
  float* vq = reinterpret_cast<float*>(scr + (size_t)(K + 2) * B);  // directions, K x B

  reduce_k1(p, part, A);
  const df N = A.get(B + K + 1, B + K + 1);
  const df invN = df_recip(N);
  // the statistics kernel's split of this pass: along mu0f with offset 1 for
  // one direction (the tensor-core form), along the initial directions q_k
  // with their offsets c_k otherwise
  for (int q = tid; q < K * B; q += kThreads)
    vq[q] = K == 1 ? p.mu0f[pb + q] : p.pilot[(size_t)part * K * B + q];
  __syncthreads();
  for (int b = tid; b < B; b += kThreads) {
    const df mf{p.mu0f[pb + b], 0.f};
    const df mk = ldf(p.muk, pb + b);
    df w{0.f, 0.f};
    for (int k = 0; k < K; ++k) {
      const float ck = K == 1 ? 1.f : p.pilot_c[(size_t)part * K + k];
      w = df_fma(df{ck, 0.f}, df{vq[k * B + b], 0.f}, w);
    }
    u1[b] = mf;
    u2[b] = ldf(p.tprev, pb + b);
    u3[b] = df_sub(w, mk);
    vd[b] = df_sub(mk, mf);
  }
  __syncthreads();
  assemble(p, A, vq, u2, u3, invN, nullptr, scr);
  if (!chol_inv_df(A, B, invd)) {
    fail_partition(p, part, false);
    return;
  }
  xtx_apply_df(A, B, invd, u2, scr, vz);
  const df q = block_dot_df(u2, vz, B, red);
  const df muv = block_dot_df(u1, vz, B, red);
  const df coff = block_dot_df(vd, vz, B, red);
  for (int b = tid; b < B; b += kThreads) p.vf[pb + b] = df_to_float(vz[b]);
  if (tid == 0) {
    float4* ps = reinterpret_cast<float4*>(p.pscal) + part;
    const float4 old = *ps;
    *ps = make_float4(df_to_float(q), df_to_float(muv), df_to_float(coff), old.w);
    p.dscal[(size_t)part * 4 + DS_Q] = df_to_double(q);
    if (!(q.hi > 0.f) || !df_isfinite(q)) p.status[part] = MF_ERR_NOT_SPD;
  }
}

// Initial background statistics only (Fig. 1 initialisation): reduce the
// statistics kernel's moments and write mu^0 and C^0 as float64 to caller
// buffers mu_out (P, B) and cov_out (P, B, B).  N <= B gives NaN.
__global__ void __launch_bounds__(kThreads) background_kernel(Params p, double* mu_out,
                                                              double* cov_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int part = blockIdx.x;
  const int tid = threadIdx.x;
  const int B = p.B, BA = p.BA, K = p.K;
  const size_t pb = (size_t)part * B;
  const DfMat A{reinterpret_cast<float*>(smem_raw), BA, BA * BA};
  df* vmu = reinterpret_cast<df*>(smem_raw) + (size_t)BA * BA;
  df* vu3 = vmu + B;
  df* scr = vu3 + B;  // (K + 2) B: assemble's scratch
  float* vq = reinterpret_cast<float*>(scr + (size_t)(K + 2) * B);
  double* cov = cov_out + (size_t)part * B * B;
  if (p.status[part] != MF_OK) {
    for (int idx = tid; idx < B * B; idx += kThreads) cov[idx] = __longlong_as_double(0x7ff8000000000000LL);
    for (int b = tid; b < B; b += kThreads) mu_out[pb + b] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  reduce_k1(p, part, A);
  const df N = A.get(B + K + 1, B + K + 1);
  const bool enough = N.hi > (float)B;
  const df invN = enough ? df_recip(N) : df{0.f, 0.f};
  init_mean(p, part, A, invN, vq, vmu, vu3);
  assemble(p, A, vq, nullptr, vu3, invN, cov, scr);
  for (int b = tid; b < B; b += kThreads)
    mu_out[pb + b] = enough ? df_to_double(vmu[b]) : __longlong_as_double(0x7ff8000000000000LL);
  if (!enough)
    for (int idx = tid; idx < B * B; idx += kThreads) cov[idx] = __longlong_as_double(0x7ff8000000000000LL);
}

size_t background_smem_bytes(int B, int BA) {
  const int K = BA - B;
  return ((size_t)BA * BA + (2 + K + 2) * (size_t)B) * sizeof(df) + (size_t)K * B * sizeof(float) +
         64;
}
cudaError_t background_set_attributes(size_t smem) {
  return cudaFuncSetAttribute(background_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}
void background_launch(size_t smem, cudaStream_t s, const Params& p, double* mu, double* cov) {
  background_kernel<<<p.P, kThreads, smem, s>>>(p, mu, cov);
}

cudaError_t solve_set_attributes(size_t s_init, size_t s_iter, size_t s_lit) {
  cudaError_t e = cudaFuncSetAttribute(solve_init_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_init);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(solve_iter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)s_iter);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(solve_literal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)s_lit);
}

// After the last pixel pass k: add its per-pixel objective terms (moment
// slot B + 3 of the pass's per-CTA partials) to the energy of iterate k.
// One warp per partition, fixed order.
__global__ void energy_final_kernel(Params p, int k) {
  const int part = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (part >= p.P || p.status[part] != MF_OK) return;
  const int K3E = k3_entries(p.B);
  const LineInfo& line = p.lines[part_line(p, part)];
  const int nunits = part_ncols(p, part) * line.n_rb;
  const float* P0 = p.k3part + (size_t)(line.k3u0 + (long long)part_col0(p, part) * line.n_rb) * K3E;
  df s{0.f, 0.f};
  for (int u = lane; u < nunits; u += 32) s = df_addf(s, P0[(size_t)u * K3E + p.B + 3]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = df_add(s, df_shfl_xor(s, o));
  if (lane == 0) p.energy[(size_t)part * p.energy_stride + k] += df_to_double(s);
}
void energy_final_launch(cudaStream_t s, const Params& p, int k) {
  energy_final_kernel<<<(p.P + 3) / 4, 128, 0, s>>>(p, k);
}

void solve_init_launch(size_t smem, cudaStream_t s, const Params& p) {
  launch_kernel(solve_init_kernel, p.P, kThreads, smem, s, p.pdl != 0, p);
}
void solve_iter_launch(size_t smem, cudaStream_t s, const Params& p, int mode, int pass) {
  launch_kernel(solve_iter_kernel, p.P, kThreads, smem, s, p.pdl != 0, p, mode, pass);
}
void solve_literal_launch(size_t smem, cudaStream_t s, const Params& p, int pass) {
  launch_kernel(solve_literal_kernel, p.P, kThreads, smem, s, p.pdl != 0, p, pass);
}

}  // namespace mf
