// Oracle (test infrastructure only): Butcher tableaux of the explicit Runge-Kutta pairs the
// paper uses (Sec. 2.2): Tsit5 (Tsitouras 2011), Dopri5 (Dormand & Prince 1980) and Verner's
// efficient 7(6) pair ("Verner 7", Verner 2010). The paper names the methods but prints no
// coefficients; the values below are those of the cited primary publications, written as the
// decimal or rational numbers those publications give. The test suite pins them against the
// Butcher order conditions, so a mistyped entry fails a test.
//
// Layout: A is s x s, row-major, strictly lower triangular; b are the weights of the
// propagated solution (order nu), bh the weights of the embedded solution (order nu-1);
// c the nodes. Dense output (Appendix A, Eq. dense) is given by weight polynomials b_j(sigma).
#pragma once

namespace orc {

enum { M_TSIT5 = 0, M_DOPRI5 = 1, M_VERN7 = 2 };

struct Tableau {
  int s;         // number of stages
  int order;     // nu, the order of the propagated solution
  bool fsal;     // last stage equals f at the new state (first stage of the next step)
  double A[10][10];
  double b[10];
  double bh[10];
  double c[10];
};

// ---- Tsit5: Tsitouras (2011), 7 stages, order 5(4), FSAL ------------------------------
inline Tableau tsit5() {
  Tableau T = {};
  T.s = 7; T.order = 5; T.fsal = true;
  double c[7] = {0.0, 0.161, 0.327, 0.9, 0.9800255409045097, 1.0, 1.0};
  for (int i = 0; i < 7; i++) T.c[i] = c[i];
  T.A[1][0] = 0.161;
  T.A[2][0] = -0.008480655492356989;  T.A[2][1] = 0.335480655492357;
  T.A[3][0] = 2.897153057105493;      T.A[3][1] = -6.359448489975075;
  T.A[3][2] = 4.3622954328695815;
  T.A[4][0] = 5.325864828439257;      T.A[4][1] = -11.748883564062828;
  T.A[4][2] = 7.4955393428898365;     T.A[4][3] = -0.09249506636175525;
  T.A[5][0] = 5.86145544294642;       T.A[5][1] = -12.92096931784711;
  T.A[5][2] = 8.159367898576159;      T.A[5][3] = -0.071584973281401;
  T.A[5][4] = -0.028269050394068383;
  T.A[6][0] = 0.09646076681806523;    T.A[6][1] = 0.01;
  T.A[6][2] = 0.4798896504144996;     T.A[6][3] = 1.379008574103742;
  T.A[6][4] = -3.290069515436081;     T.A[6][5] = 2.324710524099774;
  for (int j = 0; j < 6; j++) T.b[j] = T.A[6][j];
  T.b[6] = 0.0;
  // The publication lists the error weights b - bh; bh follows from them.
  double btilde[7] = {-0.00178001105222577714, -0.0008164344596567469, 0.007880878010261995,
                      -0.1447110071732629,     0.5823571654525552,    -0.45808210592918697,
                      0.015151515151515152};
  for (int j = 0; j < 7; j++) T.bh[j] = T.b[j] - btilde[j];
  return T;
}

// ---- Dopri5: Dormand & Prince (1980), 7 stages, order 5(4), FSAL ------------------------
inline Tableau dopri5() {
  Tableau T = {};
  T.s = 7; T.order = 5; T.fsal = true;
  double c[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
  for (int i = 0; i < 7; i++) T.c[i] = c[i];
  T.A[1][0] = 1.0 / 5;
  T.A[2][0] = 3.0 / 40;           T.A[2][1] = 9.0 / 40;
  T.A[3][0] = 44.0 / 45;          T.A[3][1] = -56.0 / 15;         T.A[3][2] = 32.0 / 9;
  T.A[4][0] = 19372.0 / 6561;     T.A[4][1] = -25360.0 / 2187;    T.A[4][2] = 64448.0 / 6561;
  T.A[4][3] = -212.0 / 729;
  T.A[5][0] = 9017.0 / 3168;      T.A[5][1] = -355.0 / 33;        T.A[5][2] = 46732.0 / 5247;
  T.A[5][3] = 49.0 / 176;         T.A[5][4] = -5103.0 / 18656;
  T.A[6][0] = 35.0 / 384;         T.A[6][1] = 0.0;                T.A[6][2] = 500.0 / 1113;
  T.A[6][3] = 125.0 / 192;        T.A[6][4] = -2187.0 / 6784;     T.A[6][5] = 11.0 / 84;
  for (int j = 0; j < 6; j++) T.b[j] = T.A[6][j];
  T.b[6] = 0.0;
  double bh[7] = {5179.0 / 57600, 0.0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200,
                  187.0 / 2100, 1.0 / 40};
  for (int j = 0; j < 7; j++) T.bh[j] = bh[j];
  return T;
}

// ---- Verner 7: Verner's efficient 7(6) pair, 10 stages, not FSAL ------------------------
inline Tableau vern7() {
  Tableau T = {};
  T.s = 10; T.order = 7; T.fsal = false;
  double c[10] = {0.0, 0.005, 0.10888888888888888, 0.16333333333333333, 0.4555,
                  0.6095094489978381, 0.884, 0.925, 1.0, 1.0};
  for (int i = 0; i < 10; i++) T.c[i] = c[i];
  T.A[1][0] = 0.005;
  T.A[2][0] = -1.07679012345679;      T.A[2][1] = 1.185679012345679;
  T.A[3][0] = 0.04083333333333333;    T.A[3][2] = 0.1225;
  T.A[4][0] = 0.6389139236255726;     T.A[4][2] = -2.455672638223657;
  T.A[4][3] = 2.272258714598084;
  T.A[5][0] = -2.6615773750187572;    T.A[5][2] = 10.804513886456137;
  T.A[5][3] = -8.3539146573962;       T.A[5][4] = 0.820487594956657;
  T.A[6][0] = 6.067741434696772;      T.A[6][2] = -24.711273635911088;
  T.A[6][3] = 20.427517930788895;     T.A[6][4] = -1.9061579788166472;
  T.A[6][5] = 1.006172249242068;
  T.A[7][0] = 12.054670076253203;     T.A[7][2] = -49.75478495046899;
  T.A[7][3] = 41.142888638604674;     T.A[7][4] = -4.461760149974004;
  T.A[7][5] = 2.042334822239175;      T.A[7][6] = -0.09834843665406107;
  T.A[8][0] = 10.138146522881808;     T.A[8][2] = -42.6411360317175;
  T.A[8][3] = 35.76384003992257;      T.A[8][4] = -4.3480228403929075;
  T.A[8][5] = 2.0098622683770357;     T.A[8][6] = 0.3487490460338272;
  T.A[8][7] = -0.27143900510483127;
  T.A[9][0] = -45.030072034298676;    T.A[9][2] = 187.3272437654589;
  T.A[9][3] = -154.02882369350186;    T.A[9][4] = 18.56465306347536;
  T.A[9][5] = -7.141809679295079;     T.A[9][6] = 1.3088085781613787;
  double b[10] = {0.04715561848627222, 0.0, 0.0, 0.25750564298434153, 0.26216653977412624,
                  0.15216092656738558, 0.4939969170032485, -0.29430311714032503,
                  0.08131747232495111, 0.0};
  double bh[10] = {0.044608606606341174, 0.0, 0.0, 0.26716403785713727, 0.22010183001772932,
                   0.2188431703143157, 0.22898717054112028, 0.0, 0.0, 0.02029518466335628};
  for (int j = 0; j < 10; j++) { T.b[j] = b[j]; T.bh[j] = bh[j]; }
  return T;
}

inline Tableau get_tableau(int method) {
  if (method == M_TSIT5) return tsit5();
  if (method == M_DOPRI5) return dopri5();
  return vern7();
}

// Dense-output weights b_j(sigma) (Appendix A, Eq. dense) for the two 5th-order pairs.
// Tsit5: the continuous extension printed with the method by Tsitouras (2011), in factored form.
// Dopri5: the 4th-order continuous extension of Dormand & Prince published with DOPRI5
// (Hairer, Norsett & Wanner, Sec. II.6), written as Hermite terms plus one correction vector.
// Verner 7 has no polynomial here: the paper re-runs a shortened step instead (Appendix A).
inline bool dense_weights(int method, double th, double* w) {
  if (method == M_TSIT5) {
    w[0] = -1.0530884977290216 * th * (th - 1.3299890189751412) *
           (th * th - 1.4364028541716351 * th + 0.7139816917074209);
    w[1] = 0.1017 * th * th * (th * th - 2.1966568338249754 * th + 1.2949852507374631);
    w[2] = 2.490627285651252793 * th * th * (th * th - 2.38535645472061657 * th + 1.57803468208092486);
    w[3] = -16.54810288924490272 * (th - 1.21712927295533244) * (th - 0.61620406037800089) * th * th;
    w[4] = 47.37952196281928122 * (th - 1.203071208372362603) * (th - 0.658047292653547382) * th * th;
    w[5] = -34.87065786149660974 * (th - 1.2) * (th - 0.666666666666666667) * th * th;
    w[6] = 2.5 * (th - 1.0) * (th - 0.6) * th * th;
    return true;
  }
  if (method == M_DOPRI5) {
    Tableau T = dopri5();
    double d[7] = {-12715105075.0 / 11282082432.0, 0.0, 87487479700.0 / 32700410799.0,
                   -10690763975.0 / 1880347072.0, 701980252875.0 / 199316789632.0,
                   -1453857185.0 / 822651844.0, 69997945.0 / 29380423.0};
    double t1 = 1.0 - th;
    for (int j = 0; j < 7; j++) {
      double e1 = (j == 0) ? 1.0 : 0.0;
      double e7 = (j == 6) ? 1.0 : 0.0;
      // y(t+th h) = y + th*D + th*t1*(h k1 - D) + th^2*t1*(2D - h k1 - h k7) + th^2*t1^2*h*sum d_j k_j,
      // with D = y1 - y = h sum b_j k_j.
      w[j] = th * T.b[j] + th * t1 * (e1 - T.b[j]) + th * th * t1 * (2.0 * T.b[j] - e1 - e7) +
             th * th * t1 * t1 * d[j];
    }
    return true;
  }
  return false;
}

}  // namespace orc
