// Wave speeds and backward explicit Runge-Kutta departure points (device, FP64).
//
// Departure point of the characteristic arriving at (x, t_{n+1}) (Sec. 2.1, eq. (depart_ODE);
// Sec. 4.1, eq. (SL2D_char1-2)): one ERK step of size -dt on d xi/dt = alpha(xi, t).  The
// paper's tableaux come from a thesis that is not part of it; this library uses forward Euler
// (r = 1), Kutta's third-order method (r = 3) and Butcher's six-stage fifth-order method (r = 5).
#pragma once

#include "common.cuh"

namespace mgrit {

struct WaveParams {
  int kind;  // mgrit_wave_kind
  double a, k, a2;
};

// alpha(x, t) of the 1D families.
MGRIT_D double alpha_1d(const WaveParams& w, double x, double t) {
  switch (w.kind) {
    case 0: return w.a;
    case 1: return cos(kTwoPi * t);
    case 2: return cos(kTwoPi * t) * cos(kTwoPi * x);
    default: return 1.0 + w.a * sin(kTwoPi * w.k * x) * cos(kTwoPi * t);
  }
}

// (alpha, beta)(x, y, t) of the 2D families.
MGRIT_D void velocity_2d(const WaveParams& w, double x, double y, double t, double& vx, double& vy) {
  switch (w.kind) {
    case 10: vx = w.a; vy = w.a2; return;
    case 11: {
      const double ct = cos(kTwoPi * t / 3.4);
      const double sy = sin(kPi * y), cx = cos(kPi * x);
      vx = sy * sy * ct;
      vy = -cx * cx * ct;
      return;
    }
    default:
      vx = 1.0 + w.a * sin(kTwoPi * y) * cos(kTwoPi * t);
      vy = 1.0 + w.a * cos(kTwoPi * x) * sin(kTwoPi * t);
      return;
  }
}

// Butcher tableau (A strictly lower triangular, b, c) of the order-r ERK, r in {1, 3, 5}.
struct Tableau {
  int stages;
  double A[6][6];
  double b[6];
  double c[6];
};

MGRIT_HD Tableau make_tableau(int r) {
  Tableau T = {};
  if (r == 1) {
    T.stages = 1;
    T.b[0] = 1.0;
  } else if (r == 3) {  // Kutta (1901), third order
    T.stages = 3;
    T.A[1][0] = 0.5;
    T.A[2][0] = -1.0;
    T.A[2][1] = 2.0;
    T.b[0] = 1.0 / 6.0;
    T.b[1] = 2.0 / 3.0;
    T.b[2] = 1.0 / 6.0;
    T.c[1] = 0.5;
    T.c[2] = 1.0;
  } else {  // Butcher (1964), six stages, fifth order, nodes 0, 1/4, 1/4, 1/2, 3/4, 1
    T.stages = 6;
    T.A[1][0] = 0.25;
    T.A[2][0] = 0.125;
    T.A[2][1] = 0.125;
    T.A[3][1] = -0.5;
    T.A[3][2] = 1.0;
    T.A[4][0] = 3.0 / 16.0;
    T.A[4][3] = 9.0 / 16.0;
    T.A[5][0] = -3.0 / 7.0;
    T.A[5][1] = 2.0 / 7.0;
    T.A[5][2] = 12.0 / 7.0;
    T.A[5][3] = -12.0 / 7.0;
    T.A[5][4] = 8.0 / 7.0;
    T.b[0] = 7.0 / 90.0;
    T.b[2] = 32.0 / 90.0;
    T.b[3] = 12.0 / 90.0;
    T.b[4] = 32.0 / 90.0;
    T.b[5] = 7.0 / 90.0;
    T.c[1] = 0.25;
    T.c[2] = 0.25;
    T.c[3] = 0.5;
    T.c[4] = 0.75;
    T.c[5] = 1.0;
  }
  return T;
}

// 2D displacement (x - xi, y - eta) of the backward ERK step.
MGRIT_D void erk_displacement_2d(const WaveParams& w, const Tableau& T, double x, double y, double t1, double dt,
                                 double& dx, double& dy) {
  double kx[6], ky[6];
  for (int s = 0; s < T.stages; ++s) {
    double xs = x, ys = y;
    for (int j = 0; j < s; ++j)
      if (T.A[s][j] != 0.0) {
        xs = xs - dt * T.A[s][j] * kx[j];
        ys = ys - dt * T.A[s][j] * ky[j];
      }
    velocity_2d(w, xs, ys, t1 - T.c[s] * dt, kx[s], ky[s]);
  }
  double sx = 0.0, sy = 0.0;
  for (int s = 0; s < T.stages; ++s)
    if (T.b[s] != 0.0) {
      sx = sx + T.b[s] * kx[s];
      sy = sy + T.b[s] * ky[s];
    }
  dx = dt * sx;
  dy = dt * sy;
}

}  // namespace mgrit
