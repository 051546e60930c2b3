// Re-injection of the particles absorbed on a wall, on the tagged injection
// faces (one thread per particle slot; only absorbed slots do work).
//
// A particle whose walk ended on an absorbing wall is replaced in its slot by
// a fresh sample of its species' injector, drawn from a counter-based
// generator so that the result does not depend on the order of the particles
// in memory:
//   u_d = top 53 bits of SplitMix64(seed, counter) * 2^-53,
//   counter = (step << 40) + (particle id << 6) + d,
// where SplitMix64(seed, c) is the output function of Steele, Lea and Flood's
// SplitMix64 applied to the state seed + (c + 1) * 0x9E3779B97F4A7C15.
// Draw 0 picks the face with probability proportional to its area (the first
// face whose running area sum exceeds u_0 times the total), draws 1 and 2 a
// uniform point on it (reflected into the lower triangle when u_1 + u_2 > 1),
// draws 3..38 the velocity: drift + sigma (sum of twelve uniforms - 6) per
// component (Irwin-Hall).  Every operation is rounded separately, whatever the
// precision mode of the particle kernel, and the new charge q w W0(x) is added
// to rho.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace fempic {
namespace dev {

constexpr int kInjectDraws = 39;

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform53(uint64_t seed, uint64_t c) {
  return __dmul_rn((double)(splitmix64(seed, c) >> 11), 1.0 / 9007199254740992.0);
}

struct InjectArgs {
  int64_t n;
  double* x[3];
  double* v[3];
  int32_t* tet;
  const uint8_t* absorbed;
  const int32_t* pid;  // particle id of each device slot
  const double* geom;
  const int32_t* dof0;
  double* rho;
  const double* face_xyz;  // [F][3][3]
  const int32_t* face_tet;
  const double* face_cum;
  int32_t n_faces;
  uint64_t seed;
  uint64_t step;
  SpeciesTable sp;  // charge q w of each species (sp.n >= 1)
  double drift[kMaxSpecies][3];
  double sigma[kMaxSpecies][3];
  unsigned long long* count;
};

template <int P>
__global__ void __launch_bounds__(256) k_inject(InjectArgs a) {
  constexpr int N0 = Nloc<P>::n0;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n || !a.absorbed[i]) return;
  using Ar = Strict;
  const uint64_t id = (uint64_t)(uint32_t)__ldg(a.pid + i);
  const uint64_t base = (a.step << 40) + (id << 6);
  const int k = species_of(a.sp, (int32_t)id);
  // face: first running sum above u_0 times the total
  const double target = Ar::mul(uniform53(a.seed, base + 0), a.face_cum[a.n_faces - 1]);
  int lo = 0, hi = a.n_faces;  // first index with cum > target in [lo, hi)
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a.face_cum[mid] > target)
      hi = mid;
    else
      lo = mid + 1;
  }
  const int f = lo < a.n_faces ? lo : a.n_faces - 1;
  double u1 = uniform53(a.seed, base + 1), u2 = uniform53(a.seed, base + 2);
  if (Ar::add(u1, u2) > 1.0) {
    u1 = Ar::sub(1.0, u1);
    u2 = Ar::sub(1.0, u2);
  }
  const double* A = a.face_xyz + (size_t)f * 9;
  double x[3], v[3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    x[c] = Ar::add(Ar::add(A[c], Ar::mul(u1, Ar::sub(A[3 + c], A[c]))), Ar::mul(u2, Ar::sub(A[6 + c], A[c])));
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double g = 0.0;
    for (int m = 0; m < 12; ++m) g = Ar::add(g, uniform53(a.seed, base + 3 + 12 * c + m));
    v[c] = Ar::add(a.drift[k][c], Ar::mul(a.sigma[k][c], Ar::sub(g, 6.0)));
  }
  const int32_t T = a.face_tet[f];
  TetGeom G;
  load_geom(a.geom, T, G);
  double l[4];
  bary<Ar>(G, x, l);
  deposit_rho<P, Ar>(l, a.sp.qw[k], a.dof0 + (size_t)T * N0, a.rho);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a.x[c][i] = x[c];
    a.v[c][i] = v[c];
  }
  a.tet[i] = T;
  atomicAdd(a.count, 1ull);
}

}  // namespace dev
}  // namespace fempic
