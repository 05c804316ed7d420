// Forward photon transport of the comparison tracer (Collin,
// arXiv:1811.04156, appendix "Ray tracer"): one photon from the point source
// through the medium to the first sensor crossing.  Shared by every tracer
// kernel of the library (pmc_trace, pmc_trace_lengths, pmc_trace_paths, the
// chain seeding and the allocation-free pmc_trace_noalloc), so there is one
// copy of the photon's physics.
//
// Transport model: the photon leaves the source in a direction drawn from the
// emission law.  Each flight draws an optical depth tau ~ Exp(1) for the next
// scattering; the next event is whichever comes first of the scattering point
// (where the scattering depth along the ray reaches tau) and the first
// crossing of the sensor sphere.  The flight's absorption depth lowers the
// photon's log weight ln w (w = exp(-integrated absorption), starting at
// w = 1).  At the sensor the photon is detected with weight w rho.  Otherwise
// it scatters (cos theta from the phase function, azimuth uniform) unless
// it started the flight farther than r_reject from the sensor centre or has
// used its max_scatter scatterings.
//
// Random numbers: Philox4x32-10 with key (k0, k1) and counter (photon low,
// photon high, i, PUR_TRACE): block i = 0 gives the emission direction
// (x, y), block i + 1 the flight after i scatterings (x: optical depth, y:
// cos theta, z: azimuth, w: the phase-mixture choice; y doubles as the
// thinning uniform of a detected photon).
#pragma once

#include "pmc_internal.h"

namespace pmc {

// Distance along direction (0, 0, nz) component nz from height z_abs at
// which the scattering depth reaches tau: tau / b in a homogeneous medium;
// layered media walk the horizontal layers the ray crosses.
__device__ inline float free_path(const DMedium& M, float z_abs, float nz, float tau) {
  if (M.kind == 0) return tau / M.b;
  float walked = 0.f, z = z_abs;
  int l = layer_of(M, z);
  for (int guard = 0; guard < (1 << 16); ++guard) {
    const float b = __ldg(M.lb + l);
    // distance to the layer's boundary in the ray's vertical direction (end
    // layers extend to infinity)
    float to_edge = __int_as_float(0x7f800000);
    int next = l;
    if (nz > 0.f && l < M.n_layers - 1) {
      to_edge = (M.z0 + (l + 1) * M.dz - z) / nz;
      next = l + 1;
    } else if (nz < 0.f && l > 0) {
      to_edge = (M.z0 + l * M.dz - z) / nz;
      next = l - 1;
    }
    to_edge = fmaxf(to_edge, 0.f);
    if (tau <= b * to_edge) return walked + tau / b;
    tau -= b * to_edge;
    walked += to_edge;
    z += to_edge * nz;
    l = next;
  }
  return walked;
}

// Distance along unit direction nh from x to the first crossing of the sphere
// |p - c|^2 = R2 ahead of x (infinity when the ray misses it).
__device__ inline float sphere_crossing(float3 x, float3 nh, float3 c, float R2) {
  const float3 w = x - c;
  const float half_b = dot(w, nh);
  const float disc = half_b * half_b - (dot(w, w) - R2);
  if (disc < 0.f) return __int_as_float(0x7f800000);
  const float t = -half_b - sqrtf(disc);
  return t > 0.f ? t : __int_as_float(0x7f800000);
}

// cos theta drawn from the phase mixture f_sl p_SL + (1 - f_sl) p_HG by
// inversion of each component's CDF (umix picks the component).
__device__ inline float draw_cos_theta(const DMedium& M, float u, float umix) {
  if (M.f_sl > 0.f && umix < M.f_sl) {
    // simplified Liu: density proportional to (1 + cos)^alpha
    return 2.0f * powf(u, 1.0f / (M.sl_alpha + 1.0f)) - 1.0f;
  }
  const float g = M.g;
  if (fabsf(g) < 1e-6f) return 2.0f * u - 1.0f;
  const float q = (1.0f - g * g) / (1.0f - g + 2.0f * g * u);
  return fminf(fmaxf((1.0f + g * g - q * q) / (2.0f * g), -1.0f), 1.0f);
}

// Unit vector at polar cosine ct and azimuth (sin, cos) = (sp, cp) about axis.
__device__ inline float3 turn_about(float3 axis, float ct, float sp, float cp) {
  float3 e1, e2;
  onb(axis, e1, e2);
  const float st = sqrtf(fmaxf(0.f, 1.0f - ct * ct));
  return ct * axis + st * (cp * e1 + sp * e2);
}

struct PhotonResult {
  bool hit;     // reached the sensor
  float lw;     // ln(w rho) of a detected photon
  float L;      // path length of a detected photon
  int nsc;      // scatterings before detection
  float u_acc;  // spare uniform of the detecting flight (thinning by w rho)
};

// One photon (index ph); with kRecord the vertices (source, scattering
// points, sensor crossing) go to (ox, oy, oz) in absolute coordinates
// (frame coordinates + S.org).
template <bool kRecord>
__device__ inline PhotonResult trace_photon(const DMedium& M, const DPair& S, uint32_t k0, uint32_t k1,
                                            unsigned long long ph, float r_reject, int max_scatter, float* ox,
                                            float* oy, float* oz) {
  const uint32_t plo = static_cast<uint32_t>(ph), phi = static_cast<uint32_t>(ph >> 32);
  const float3 c = f3(S.c[0], S.c[1], S.c[2]);
  const float3 org = f3(S.org[0], S.org[1], S.org[2]);
  auto record = [&](int i, float3 p) {
    if constexpr (kRecord) {
      ox[i] = p.x + org.x;
      oy[i] = p.y + org.y;
      oz[i] = p.z + org.z;
    }
  };
  // emission: isotropic, or von Mises-Fisher about S.dir (inverse CDF in cos)
  float3 nh;
  {
    const uint4 r = philox4x32_10(make_uint4(plo, phi, 0u, PUR_TRACE), k0, k1);
    float sp, cp;
    sincospif(2.0f * u01(r.y), &sp, &cp);
    const float u0 = u01(r.x);
    if (S.emission != 0) {
      const float ct = 1.0f + logf(fmaf(1.0f - u0, expf(-2.0f * S.kappa), u0)) / S.kappa;
      nh = turn_about(f3(S.dir[0], S.dir[1], S.dir[2]), ct, sp, cp);
    } else {
      const float ct = 2.0f * u0 - 1.0f;
      const float st = sqrtf(fmaxf(0.f, 1.0f - ct * ct));
      nh = f3(st * cp, st * sp, ct);
    }
  }
  float3 x = f3(0.f, 0.f, 0.f);
  record(0, x);
  float lnw = 0.f, walked = 0.f;
  PhotonResult res{false, 0.f, 0.f, 0, 1.f};
  for (int i = 0;; ++i) {
    const uint4 r = philox4x32_10(make_uint4(plo, phi, static_cast<uint32_t>(i + 1), PUR_TRACE), k0, k1);
    const float to_scatter = free_path(M, x.z + S.zoff, nh.z, -logf(u01(r.x)));
    const float to_sensor = sphere_crossing(x, nh, c, S.R2);
    const bool detect = to_sensor < to_scatter;
    const float flight = detect ? to_sensor : to_scatter;
    const float3 next = x + flight * nh;
    float ta, tb;
    seg_tau(M, x.z + S.zoff, next.z + S.zoff, flight, ta, tb);
    lnw -= ta;
    record(i + 1, next);
    if (detect) {
      float lr = 0.f;
      if (S.rho != 0) {
        const float xx = dot(sensor_normal(S, next), f3(S.rho_hat[0], S.rho_hat[1], S.rho_hat[2]));
        lr = fmaf(3.0f, xx, -1.0f) - logf(coshf(fmaf(2.0f, xx, 0.7f)));
      }
      res = PhotonResult{true, lnw + lr, walked + to_sensor, i, u01(r.y)};
      return res;
    }
    const float3 from_c = x - c;
    const bool escaped = dot(from_c, from_c) > r_reject * r_reject;
    if (escaped || i == max_scatter) return res;
    x = next;
    walked += to_scatter;
    float sp, cp;
    sincospif(2.0f * u01(r.z), &sp, &cp);
    nh = turn_about(nh, draw_cos_theta(M, u01(r.y), u01(r.w)), sp, cp);
    nh = rsqrtf(dot(nh, nh)) * nh;
  }
}

}  // namespace pmc
