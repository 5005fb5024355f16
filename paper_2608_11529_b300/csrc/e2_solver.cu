// C ABI: reference states by block Davidson on the device, with a host
// Jacobi eigensolver for the small projected problem.
#include "e2_host.h"


namespace e2 {

using cd = std::complex<double>;

// Cyclic Jacobi for a complex Hermitian matrix A (n x n, row-major):
// eigenvalues ascending in w, eigenvectors in the columns of V (row-major).
// Each rotation U = [[c, s e^{i phi}], [-s e^{-i phi}, c]] in the (p,q) plane
// zeroes A_pq = g e^{i phi}: t = s/c solves t^2 + 2 tau t - 1 = 0,
// tau = (A_qq - A_pp) / (2 g), smaller root.
void herm_eig(int n, std::vector<cd> A, std::vector<double>& w, std::vector<cd>& V) {
  V.assign((size_t)n * n, cd(0.0, 0.0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int p = 0; p < n; ++p) {
      dia += std::norm(A[(size_t)p * n + p]);
      for (int q = p + 1; q < n; ++q) off += std::norm(A[(size_t)p * n + q]);
    }
    if (off <= 1e-32 * (dia + 1e-300)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const cd apq = A[(size_t)p * n + q];
        const double g = std::abs(apq);
        if (g < 1e-300) continue;
        const cd ph = apq / g;
        const double a = A[(size_t)p * n + p].real(), bq = A[(size_t)q * n + q].real();
        const double tau = (bq - a) / (2.0 * g);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        const cd u00 = cs, u01 = sn * ph, u10 = -sn * std::conj(ph), u11 = cs;
        for (int r = 0; r < n; ++r) {  // A <- A U, V <- V U
          cd x = A[(size_t)r * n + p], y = A[(size_t)r * n + q];
          A[(size_t)r * n + p] = x * u00 + y * u10;
          A[(size_t)r * n + q] = x * u01 + y * u11;
          x = V[(size_t)r * n + p];
          y = V[(size_t)r * n + q];
          V[(size_t)r * n + p] = x * u00 + y * u10;
          V[(size_t)r * n + q] = x * u01 + y * u11;
        }
        for (int r = 0; r < n; ++r) {  // A <- U^H A
          cd x = A[(size_t)p * n + r], y = A[(size_t)q * n + r];
          A[(size_t)p * n + r] = std::conj(u00) * x + std::conj(u10) * y;
          A[(size_t)q * n + r] = std::conj(u01) * x + std::conj(u11) * y;
        }
      }
  }
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return A[(size_t)x * n + x].real() < A[(size_t)y * n + y].real(); });
  w.resize(n);
  std::vector<cd> Vs((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = A[(size_t)ord[j] * n + ord[j]].real();
    for (int i = 0; i < n; ++i) Vs[(size_t)i * n + j] = V[(size_t)i * n + ord[j]];
  }
  V.swap(Vs);
}

}  // namespace e2

using namespace e2;

extern "C" {

e2_status e2_reference_workspace_size(const e2_problem* P, size_t* bytes) {
  if (!P || !bytes) return E2_ERR_INVALID_ARG;
  *bytes = P->solve_bytes;
  return E2_OK;
}

e2_status e2_reference_solve(e2_problem* P, const e2_inputs* in, double tol, int max_iter, void* workspace,
                             size_t workspace_bytes, void* stream_, double* c_out, double* E0_out, int* iters_out) {
  if (!P || !in || !c_out || !E0_out || !in->h || !in->B_c || !in->c) return E2_ERR_INVALID_ARG;
  if (P->d.L_extra > 0 && (!in->B_x || !in->w_x)) return E2_ERR_INVALID_ARG;
  if (!(tol > 0.0) || max_iter < 1) return E2_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < P->solve_bytes || ((uintptr_t)workspace & 255)) return E2_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream_;
  unsigned char* ws = (unsigned char*)workspace;
  cudaGetLastError();
  if (setup_common(P, in, ws, st) != E2_OK) return E2_ERR_CUDA;
  const int R = P->d.n_roots, mmax = P->sv_mmax;
  const DevList LP = dev_list(P, P->listP, ws);
  const int64_t np = LP.n;
  if (np < R) return E2_ERR_SHAPE;
  Ctx X = ctx(P, ws);
  Tabs T = tables(P, ws, 0);
  double2* V = (double2*)(ws + P->o_sV);
  double2* S = (double2*)(ws + P->o_sS);
  double2* Xv = (double2*)(ws + P->o_sX);
  double2* Rv = (double2*)(ws + P->o_sR);
  double2* Dv = (double2*)(ws + P->o_sD);
  double2* Tv = (double2*)(ws + P->o_sT);
  double2* Gd = (double2*)(ws + P->o_sG);
  double2* Yd = (double2*)(ws + P->o_sY);
  const DevList L11 = dev_list(P, P->list_of[4], ws), L02 = dev_list(P, P->list_of[2], ws);
  auto sigma = [&](const double2* v, double2* s) {
    build_tables(P, ws, st, v, T, false);
    (k_sigma<<<blocks(np), 256, 0, st>>>(LP, L11, L02, P->das, X.sp, X.binom, T.DTDU, T.DTU,
                                        (const double2*)(ws + P->o_X00), X.f, s), ++g_launches);
  };
  auto gram = [&](const double2* a, int na_, const double2* bb, int nb_) {
    std::vector<cd> out((size_t)na_ * nb_);
    (k_gram<<<na_ * nb_, 256, 0, st>>>(a, bb, np, nb_, Gd), ++g_launches);
    cudaMemcpyAsync(out.data(), Gd, 16 * out.size(), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return out;
  };
  auto upload = [&](const std::vector<cd>& y) {
    cudaMemcpyAsync(Yd, y.data(), 16 * y.size(), cudaMemcpyHostToDevice, st);
  };
  int k = 0;
  // copy a vector into slot k, orthogonalise it twice against slots < k, normalise, and build its sigma
  auto append = [&](const double2* src) -> bool {
    double2* vk = V + (int64_t)k * np;
    if (src != vk) cudaMemcpyAsync(vk, src, 16 * (size_t)np, cudaMemcpyDeviceToDevice, st);
    for (int pass = 0; pass < 2 && k > 0; ++pass) {
      std::vector<cd> ov = gram(V, k, vk, 1);
      for (auto& z : ov) z = -z;
      upload(ov);
      (k_lincomb<<<dim3(blocks(np), 1), 256, 0, st>>>(V, k, np, (const double2*)Yd, 1, 1, vk), ++g_launches);
    }
    double nrm = gram(vk, 1, vk, 1)[0].real();
    if (!(nrm > 1e-24)) return false;
    (k_scale<<<blocks(np), 256, 0, st>>>(vk, np, 1.0 / std::sqrt(nrm)), ++g_launches);
    sigma(vk, S + (int64_t)k * np);
    ++k;
    return true;
  };
  for (int j = 0; j < R; ++j)
    if (!append((const double2*)in->c + (int64_t)j * np)) return E2_ERR_SHAPE;
  std::vector<double> w;
  std::vector<cd> Y;
  int it = 0;
  for (; it < max_iter; ++it) {
    std::vector<cd> H = gram(V, k, S, k);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j <= i; ++j) {
        cd a = 0.5 * (H[(size_t)i * k + j] + std::conj(H[(size_t)j * k + i]));
        H[(size_t)i * k + j] = a;
        H[(size_t)j * k + i] = std::conj(a);
      }
    herm_eig(k, H, w, Y);
    std::vector<cd> Yr((size_t)k * R);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < R; ++j) Yr[(size_t)i * R + j] = Y[(size_t)i * k + j];
    upload(Yr);
    (k_lincomb<<<dim3(blocks(np), R), 256, 0, st>>>(V, k, np, (const double2*)Yd, R, 0, Xv), ++g_launches);
    (k_lincomb<<<dim3(blocks(np), R), 256, 0, st>>>(S, k, np, (const double2*)Yd, R, 0, Rv), ++g_launches);
    for (int j = 0; j < R; ++j)
      (k_residual<<<blocks(np), 256, 0, st>>>(Rv + (int64_t)j * np, Xv + (int64_t)j * np, LP.eA, np, w[j],
                                             Dv + (int64_t)j * np), ++g_launches);
    std::vector<cd> rn = gram(Rv, R, Rv, R);
    bool done = true;
    std::vector<int> open;
    for (int j = 0; j < R; ++j)
      if (std::sqrt(std::max(0.0, rn[(size_t)j * R + j].real())) >= tol) {
        done = false;
        open.push_back(j);
      }
    if (done) break;
    if (k + (int)open.size() > mmax) {  // restart from the Ritz vectors
      (k_lincomb<<<dim3(blocks(np), R), 256, 0, st>>>(S, k, np, (const double2*)Yd, R, 0, Tv), ++g_launches);
      cudaMemcpyAsync(V, Xv, 16 * (size_t)R * np, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(S, Tv, 16 * (size_t)R * np, cudaMemcpyDeviceToDevice, st);
      k = R;
    }
    int added = 0;
    for (int j : open)
      if (k < mmax && append(Dv + (int64_t)j * np)) ++added;
    if (added == 0) break;
  }
  cudaMemcpyAsync(c_out, Xv, 16 * (size_t)R * np, cudaMemcpyDeviceToDevice, st);
  double EOh = 0.0;
  cudaMemcpyAsync(&EOh, X.EO, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return E2_ERR_CUDA;
  for (int j = 0; j < R; ++j) E0_out[j] = w[j] + EOh;
  if (iters_out) *iters_out = it;
  return E2_OK;
}

}  // extern "C"
