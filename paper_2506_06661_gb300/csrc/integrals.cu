// s-type Gaussian integrals: Boys entry point, one-electron S/T/V, the two-centre
// Coulomb metric and the three-centre tensor (Q|mn) of the density-fitting equations
// (arXiv 2506.06661, Section "Density fitting").  Products of two primitives use the
// Gaussian product theorem of the paper's overlap example: p = a + b, mu = ab/p,
// P = (aA + bB)/p.
#include "common.cuh"
#include "boys.cuh"
#include "kernels.cuh"

namespace dfscf {

__device__ __forceinline__ double norm_s(double a) {
  // (2a/pi)^(3/4)
  double x = 2.0 * a / kPi;
  return sqrt(x * sqrt(x));
}

__global__ void boys_kernel(const double* __restrict__ t, long n, double* __restrict__ out) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = boys_f0(t[i]);
}

// S_ab = N_a N_b (pi/p)^(3/2) e^{-mu R^2};  T_ab = mu (3 - 2 mu R^2) S_ab;
// V_ab = -sum_C Z_C N_a N_b (2pi/p) e^{-mu R^2} F0(p |P - C|^2).
__global__ void int1e_kernel(const double* __restrict__ xyz, const double* __restrict__ ex, int nao,
                             const double* __restrict__ nxyz, const double* __restrict__ nz, int natm,
                             double* __restrict__ S, double* __restrict__ T, double* __restrict__ V) {
  __shared__ double sn[4 * 128];
  int a = blockIdx.y;
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = b < nao;
  int bb = ok ? b : 0;
  double ea = ex[a], eb = ex[bb];
  double p = ea + eb, mu = ea * eb / p;
  double dx = xyz[3 * a] - xyz[3 * bb], dy = xyz[3 * a + 1] - xyz[3 * bb + 1], dz = xyz[3 * a + 2] - xyz[3 * bb + 2];
  double r2 = dx * dx + dy * dy + dz * dz;
  double kab = norm_s(ea) * norm_s(eb) * exp(-mu * r2);
  double px = (ea * xyz[3 * a] + eb * xyz[3 * bb]) / p;
  double py = (ea * xyz[3 * a + 1] + eb * xyz[3 * bb + 1]) / p;
  double pz = (ea * xyz[3 * a + 2] + eb * xyz[3 * bb + 2]) / p;
  double v = 0.0;
  if (V) {
    for (int c0 = 0; c0 < natm; c0 += 128) {
      __syncthreads();
      for (int c = threadIdx.x; c < 128 && c0 + c < natm; c += blockDim.x) {
        sn[4 * c] = nxyz[3 * (c0 + c)];
        sn[4 * c + 1] = nxyz[3 * (c0 + c) + 1];
        sn[4 * c + 2] = nxyz[3 * (c0 + c) + 2];
        sn[4 * c + 3] = nz[c0 + c];
      }
      __syncthreads();
      int cn = min(128, natm - c0);
      for (int c = 0; c < cn; ++c) {
        double qx = px - sn[4 * c], qy = py - sn[4 * c + 1], qz = pz - sn[4 * c + 2];
        v -= sn[4 * c + 3] * boys_f0(p * (qx * qx + qy * qy + qz * qz));
      }
    }
    v *= kab * 2.0 * kPi / p;
  }
  if (!ok) return;
  double s = kab * (kPi / p) * sqrt(kPi / p);
  size_t o = (size_t)a * nao + b;
  if (S) S[o] = s;
  if (T) T[o] = mu * (3.0 - 2.0 * mu * r2) * s;
  if (V) V[o] = v;
}

// (c|d) = N_c N_d 2 pi^{5/2} / (c d sqrt(c + d)) F0(cd/(c+d) R^2).  With omega > 0 the
// long-range operator erf(omega r)/r of the paper's LRDF split: the reduced exponent
// rho = cd/(c+d) becomes rho f in the Boys argument and the prefactor gains sqrt(f),
// f = omega^2 / (rho + omega^2).
__global__ void int2c_kernel(const double* __restrict__ xyz, const double* __restrict__ ex, int naux, double omega,
                             double* __restrict__ M) {
  int c = blockIdx.y;
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= naux) return;
  double ec = ex[c], ed = ex[d];
  double dx = xyz[3 * c] - xyz[3 * d], dy = xyz[3 * c + 1] - xyz[3 * d + 1], dz = xyz[3 * c + 2] - xyz[3 * d + 2];
  double r2 = dx * dx + dy * dy + dz * dz;
  double pre = norm_s(ec) * norm_s(ed) * 2.0 * kPi * kPi * sqrt(kPi) / (ec * ed * sqrt(ec + ed));
  double rho = ec * ed / (ec + ed);
  if (omega > 0.0) {
    const double f = omega * omega / (rho + omega * omega);
    pre *= sqrt(f);
    rho *= f;
  }
  M[(size_t)c * naux + d] = pre * boys_f0(rho * r2);
}

// Per packed pair mn: product exponent p, centre P and K_mn = N_m N_n e^{-mu R^2} 2 pi^{5/2} / p.
__global__ void pair_table_kernel(const double* __restrict__ xyz, const double* __restrict__ ex, long npair,
                                  double* __restrict__ pp, double* __restrict__ px, double* __restrict__ py,
                                  double* __restrict__ pz, double* __restrict__ pk) {
  long ij = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= npair) return;
  int a, b;
  unpack_pair(ij, a, b);
  double ea = ex[a], eb = ex[b];
  double p = ea + eb, mu = ea * eb / p;
  double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1], dz = xyz[3 * a + 2] - xyz[3 * b + 2];
  pp[ij] = p;
  px[ij] = (ea * xyz[3 * a] + eb * xyz[3 * b]) / p;
  py[ij] = (ea * xyz[3 * a + 1] + eb * xyz[3 * b + 1]) / p;
  pz[ij] = (ea * xyz[3 * a + 2] + eb * xyz[3 * b + 2]) / p;
  pk[ij] = norm_s(ea) * norm_s(eb) * exp(-mu * (dx * dx + dy * dy + dz * dz)) * 2.0 * kPi * kPi * sqrt(kPi) / p;
}

// (Q|mn) = K_mn N_Q / (c sqrt(p + c)) F0(p c / (p + c) |P - C|^2), written row Q of R
// (row stride ld, padding columns [npair, ld) set to zero).  One lane per (Q, mn).
__global__ void int3c_kernel(const double* __restrict__ pp, const double* __restrict__ px,
                             const double* __restrict__ py, const double* __restrict__ pz,
                             const double* __restrict__ pk, long npair, long ld,
                             const double* __restrict__ axyz, const double* __restrict__ aex, int q0, double omega,
                             double* __restrict__ R) {
  int q = q0 + blockIdx.y;
  long ij = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= ld) return;
  double* row = R + (size_t)q * ld;
  if (ij >= npair) {
    row[ij] = 0.0;
    return;
  }
  double c = aex[q];
  double cx = axyz[3 * q], cy = axyz[3 * q + 1], cz = axyz[3 * q + 2];
  double p = pp[ij];
  double dx = px[ij] - cx, dy = py[ij] - cy, dz = pz[ij] - cz;
  double inv = 1.0 / (p + c);
  double rho = p * c * inv;
  double pre = pk[ij] * norm_s(c) / c * sqrt(inv);
  if (omega > 0.0) {  // long-range operator, as in int2c_kernel
    const double f = omega * omega / (rho + omega * omega);
    pre *= sqrt(f);
    rho *= f;
  }
  row[ij] = pre * boys_f0(rho * (dx * dx + dy * dy + dz * dz));
}

__global__ void enuc_kernel(const double* __restrict__ xyz, const double* __restrict__ z, int natm,
                            double* __restrict__ out) {
  __shared__ double sh[32];
  double e = 0.0;
  for (long k = threadIdx.x; k < (long)natm * natm; k += blockDim.x) {
    int a = (int)(k / natm), b = (int)(k % natm);
    if (b < a) {
      double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1], dz = xyz[3 * a + 2] - xyz[3 * b + 2];
      e += z[a] * z[b] / sqrt(dx * dx + dy * dy + dz * dz);
    }
  }
  e = block_sum(e, sh);
  if (threadIdx.x == 0) *out = e;
}

int launch_int1e(const double* ao_xyz, const double* ao_exp, int nao, const double* nuc_xyz, const double* nuc_z,
                 int natm, double* S, double* T, double* V, cudaStream_t s) {
  dim3 grid((nao + 127) / 128, nao);
  int1e_kernel<<<grid, 128, 0, s>>>(ao_xyz, ao_exp, nao, nuc_xyz, nuc_z, natm, S, T, V);
  DF_LAUNCHED("int1e_kernel");
  return DF_OK;
}

int launch_int2c(const double* xyz, const double* ex, int naux, double* M, cudaStream_t s, double omega) {
  dim3 grid((naux + 127) / 128, naux);
  int2c_kernel<<<grid, 128, 0, s>>>(xyz, ex, naux, omega, M);
  DF_LAUNCHED("int2c_kernel");
  return DF_OK;
}

int launch_pair_table(const double* ao_xyz, const double* ao_exp, int nao, double* pair_tab, cudaStream_t s) {
  long npair = npair_of(nao);
  double* pp = pair_tab;
  pair_table_kernel<<<(unsigned)((npair + 255) / 256), 256, 0, s>>>(ao_xyz, ao_exp, npair, pp, pp + npair,
                                                                    pp + 2 * npair, pp + 3 * npair, pp + 4 * npair);
  DF_LAUNCHED("pair_table_kernel");
  return DF_OK;
}

int launch_int3c(const double* ao_xyz, const double* ao_exp, int nao, const double* aux_xyz, const double* aux_exp,
                 int naux, double* R, long ld, double* pair_tab, cudaStream_t s, double omega) {
  long npair = npair_of(nao);
  double* pp = pair_tab;
  double* px = pp + npair;
  double* py = px + npair;
  double* pz = py + npair;
  double* pk = pz + npair;
  DF_TRY(launch_pair_table(ao_xyz, ao_exp, nao, pair_tab, s));
  for (int q0 = 0; q0 < naux; q0 += 32768) {
    dim3 grid((unsigned)((ld + 255) / 256), (unsigned)min(32768, naux - q0));
    int3c_kernel<<<grid, 256, 0, s>>>(pp, px, py, pz, pk, npair, ld, aux_xyz, aux_exp, q0, omega, R);
    DF_LAUNCHED("int3c_kernel");
  }
  return DF_OK;
}

int launch_enuc(const double* xyz, const double* z, int natm, double* out, cudaStream_t s) {
  enuc_kernel<<<1, 256, 0, s>>>(xyz, z, natm, out);
  DF_LAUNCHED("enuc_kernel");
  return DF_OK;
}

}  // namespace dfscf

using namespace dfscf;

extern "C" int df_boys_f0(const double* t, long n, double* out, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(n >= 0, DF_ERR_ARG, "df_boys_f0: n < 0");
  if (n == 0) return DF_OK;
  DF_REQUIRE(t && out, DF_ERR_ARG, "df_boys_f0: null pointer");
  boys_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t, n, out);
  DF_LAUNCHED("boys_kernel");
  return DF_OK;
}

extern "C" int df_int1e(const double* ao_xyz, const double* ao_exp, int nao, const double* nuc_xyz,
                        const double* nuc_z, int natm, double* S, double* T, double* V, cudaStream_t s) {
  clear_error();
  DF_REQUIRE(nao > 0 && natm >= 0, DF_ERR_ARG, "df_int1e: bad sizes nao=%d natm=%d", nao, natm);
  DF_REQUIRE(ao_xyz && ao_exp, DF_ERR_ARG, "df_int1e: null basis arrays");
  DF_REQUIRE(!V || natm == 0 || (nuc_xyz && nuc_z), DF_ERR_ARG, "df_int1e: V requested without nuclei");
  return launch_int1e(ao_xyz, ao_exp, nao, nuc_xyz, nuc_z, natm, S, T, V, s);
}

extern "C" int df_nuclear_repulsion(const double* nuc_xyz, const double* nuc_z, int natm, double* e_nuc,
                                    cudaStream_t s) {
  clear_error();
  DF_REQUIRE(natm >= 0 && e_nuc, DF_ERR_ARG, "df_nuclear_repulsion: bad arguments");
  DF_REQUIRE(natm == 0 || (nuc_xyz && nuc_z), DF_ERR_ARG, "df_nuclear_repulsion: null pointer");
  return launch_enuc(nuc_xyz, nuc_z, natm, e_nuc, s);
}

DF_BOUNDS_READER(bounds_read_integrals)
