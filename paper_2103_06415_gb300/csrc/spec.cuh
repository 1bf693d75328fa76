// Spectral-step parameters of a level solve from a context (tables in the context precision).
#pragma once
#include "dst.cuh"
#include "internal.h"

// h: spacing of the level; ring: pointer to the boundary-ring spectra or NULL for zero boundary values
template <typename T>
dst::SpecParams<T> spec_params(const fsi_ctx* c, double h, const T* ring) {
  dst::SpecParams<T> sp = {};
  sp.lx = (const T*)c->lxT;
  sp.ly = (const T*)c->lyT;
  sp.sx1 = (const T*)c->sx1T;
  sp.sxN = (const T*)c->sxNT;
  sp.sy1 = (const T*)c->sy1T;
  sp.syN = (const T*)c->syNT;
  sp.ring = ring;
  sp.ring_ld = c->ring_ld;
  sp.inv_h2 = T(1.0 / (h * h));
  sp.inv_dt = T(1.0 / c->g.dt);
  sp.inv_2re = T(0.5 / c->g.re);
  sp.norm = T(4.0 / ((double)c->Mx * (double)c->My));
  sp.ring_w = T((0.5 / c->g.re) * (1.0 / (h * h)));
  sp.Mx = c->Mx;
  sp.My = c->My;
  return sp;
}
