// Device Butcher tableaux of the explicit Runge-Kutta pairs of Sec. 2.2: Tsit5 (Tsitouras 2011),
// Dopri5 (Dormand & Prince 1980) and Verner's efficient 7(6) pair. The paper names the methods
// but prints no coefficients; these are the values of the cited publications. All entries are
// compile-time constants, so after loop unrolling each coefficient is an instruction immediate
// and zero entries generate no instruction.
//
// Per method: S stages, ORDER nu, FSAL (the last stage is f at the new state), NREV the number of
// leading stages the new state depends on (the stages the adjoint has to reverse), and the dense
// output weights b_j(sigma) of Appendix A, Eq. dense where the method has them.
#pragma once

namespace gs {

struct Tsit5 {
  static constexpr int S = 7, ORDER = 5, NREV = 6;
  static constexpr bool FSAL = true, DENSE_POLY = true;
  __host__ __device__ static constexpr double c(int i) {
    constexpr double v[7] = {0.0, 0.161, 0.327, 0.9, 0.9800255409045097, 1.0, 1.0};
    return v[i];
  }
  __host__ __device__ static constexpr double a(int i, int j) {
    constexpr double A[7][6] = {
        {0, 0, 0, 0, 0, 0},
        {0.161, 0, 0, 0, 0, 0},
        {-0.008480655492356989, 0.335480655492357, 0, 0, 0, 0},
        {2.897153057105493, -6.359448489975075, 4.3622954328695815, 0, 0, 0},
        {5.325864828439257, -11.748883564062828, 7.4955393428898365, -0.09249506636175525, 0, 0},
        {5.86145544294642, -12.92096931784711, 8.159367898576159, -0.071584973281401,
         -0.028269050394068383, 0},
        {0.09646076681806523, 0.01, 0.4798896504144996, 1.379008574103742, -3.290069515436081,
         2.324710524099774}};
    return A[i][j];
  }
  __host__ __device__ static constexpr double b(int j) { return j < 6 ? a(6, j) : 0.0; }
  // error weights b - bhat, as published
  __host__ __device__ static constexpr double bt(int j) {
    constexpr double v[7] = {-0.00178001105222577714, -0.0008164344596567469, 0.007880878010261995,
                             -0.1447110071732629,     0.5823571654525552,    -0.45808210592918697,
                             0.015151515151515152};
    return v[j];
  }
  // Tsitouras' continuous extension, factored form
  template <class R>
  __device__ static void dense(R th, R* w) {
    w[0] = R(-1.0530884977290216) * th * (th - R(1.3299890189751412)) *
           (th * th - R(1.4364028541716351) * th + R(0.7139816917074209));
    w[1] = R(0.1017) * th * th * (th * th - R(2.1966568338249754) * th + R(1.2949852507374631));
    w[2] = R(2.490627285651252793) * th * th * (th * th - R(2.38535645472061657) * th + R(1.57803468208092486));
    w[3] = R(-16.54810288924490272) * (th - R(1.21712927295533244)) * (th - R(0.61620406037800089)) * th * th;
    w[4] = R(47.37952196281928122) * (th - R(1.203071208372362603)) * (th - R(0.658047292653547382)) * th * th;
    w[5] = R(-34.87065786149660974) * (th - R(1.2)) * (th - R(0.666666666666666667)) * th * th;
    w[6] = R(2.5) * (th - R(1.0)) * (th - R(0.6)) * th * th;
  }
};

struct Dopri5 {
  static constexpr int S = 7, ORDER = 5, NREV = 6;
  static constexpr bool FSAL = true, DENSE_POLY = true;
  __host__ __device__ static constexpr double c(int i) {
    constexpr double v[7] = {0.0, 0.2, 0.3, 0.8, 8.0 / 9.0, 1.0, 1.0};
    return v[i];
  }
  __host__ __device__ static constexpr double a(int i, int j) {
    constexpr double A[7][6] = {
        {0, 0, 0, 0, 0, 0},
        {1.0 / 5, 0, 0, 0, 0, 0},
        {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
        {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
        {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
        {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
        {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
    return A[i][j];
  }
  __host__ __device__ static constexpr double b(int j) { return j < 6 ? a(6, j) : 0.0; }
  __host__ __device__ static constexpr double bhat(int j) {
    constexpr double v[7] = {5179.0 / 57600, 0.0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200,
                             187.0 / 2100, 1.0 / 40};
    return v[j];
  }
  __host__ __device__ static constexpr double bt(int j) { return b(j) - bhat(j); }
  // 4th-order continuous extension published with the pair (Hairer-Norsett-Wanner I, II.6):
  // Hermite terms in (y, y1, h k1, h k7) plus sigma^2 (1-sigma)^2 h sum d_j k_j.
  __host__ __device__ static constexpr double dd(int j) {
    constexpr double v[7] = {-12715105075.0 / 11282082432.0, 0.0, 87487479700.0 / 32700410799.0,
                             -10690763975.0 / 1880347072.0, 701980252875.0 / 199316789632.0,
                             -1453857185.0 / 822651844.0, 69997945.0 / 29380423.0};
    return v[j];
  }
  template <class R>
  __device__ static void dense(R th, R* w) {
    const R t1 = R(1) - th;
#pragma unroll
    for (int j = 0; j < 7; j++) {
      const R bj = R(b(j));
      const R e1 = j == 0 ? R(1) : R(0);
      const R e7 = j == 6 ? R(1) : R(0);
      w[j] = th * bj + th * t1 * (e1 - bj) + th * th * t1 * (R(2) * bj - e1 - e7) +
             th * th * t1 * t1 * R(dd(j));
    }
  }
};

struct Vern7 {
  static constexpr int S = 10, ORDER = 7, NREV = 9;
  static constexpr bool FSAL = false, DENSE_POLY = false;
  __host__ __device__ static constexpr double c(int i) {
    constexpr double v[10] = {0.0, 0.005, 0.10888888888888888, 0.16333333333333333, 0.4555,
                              0.6095094489978381, 0.884, 0.925, 1.0, 1.0};
    return v[i];
  }
  __host__ __device__ static constexpr double a(int i, int j) {
    constexpr double A[10][9] = {
        {0, 0, 0, 0, 0, 0, 0, 0, 0},
        {0.005, 0, 0, 0, 0, 0, 0, 0, 0},
        {-1.07679012345679, 1.185679012345679, 0, 0, 0, 0, 0, 0, 0},
        {0.04083333333333333, 0, 0.1225, 0, 0, 0, 0, 0, 0},
        {0.6389139236255726, 0, -2.455672638223657, 2.272258714598084, 0, 0, 0, 0, 0},
        {-2.6615773750187572, 0, 10.804513886456137, -8.3539146573962, 0.820487594956657, 0, 0, 0, 0},
        {6.067741434696772, 0, -24.711273635911088, 20.427517930788895, -1.9061579788166472,
         1.006172249242068, 0, 0, 0},
        {12.054670076253203, 0, -49.75478495046899, 41.142888638604674, -4.461760149974004,
         2.042334822239175, -0.09834843665406107, 0, 0},
        {10.138146522881808, 0, -42.6411360317175, 35.76384003992257, -4.3480228403929075,
         2.0098622683770357, 0.3487490460338272, -0.27143900510483127, 0},
        {-45.030072034298676, 0, 187.3272437654589, -154.02882369350186, 18.56465306347536,
         -7.141809679295079, 1.3088085781613787, 0, 0}};
    return A[i][j];
  }
  __host__ __device__ static constexpr double b(int j) {
    constexpr double v[10] = {0.04715561848627222, 0.0, 0.0, 0.25750564298434153, 0.26216653977412624,
                              0.15216092656738558, 0.4939969170032485, -0.29430311714032503,
                              0.08131747232495111, 0.0};
    return v[j];
  }
  __host__ __device__ static constexpr double bhat(int j) {
    constexpr double v[10] = {0.044608606606341174, 0.0, 0.0, 0.26716403785713727, 0.22010183001772932,
                              0.2188431703143157, 0.22898717054112028, 0.0, 0.0, 0.02029518466335628};
    return v[j];
  }
  __host__ __device__ static constexpr double bt(int j) { return b(j) - bhat(j); }
  template <class R>
  __device__ static void dense(R, R*) {}
};

// The coefficients of a pair's stages in Nystrom form, for second-order systems y = (x, v),
// f = (v, a(x)). With V_l = v + h sum_m a_lm a_m, the stage positions are
//   X_j = x + h (sum_l a_jl) v + h^2 sum_m (A^2)_jm a_m,
// the new position x + h (sum_j b_j) v + h^2 sum_m (b A)_m a_m and the position error
// h (sum_j bt_j) v + h^2 sum_m (bt A)_m a_m, where sum_j b_j = 1 and sum_j bt_j = 0. A is strictly
// lower triangular, so (A^2)_jm vanishes for m >= j - 1. The same stages as the general form, with
// stage sums over three components instead of six.
template <class Tab>
struct Nystrom {
  __host__ __device__ static constexpr double row(int j) {  // sum_l a_jl
    double s = 0.0;
    for (int l = 0; l < j; l++) s += Tab::a(j, l);
    return s;
  }
  __host__ __device__ static constexpr double aa(int j, int m) {  // (A^2)_jm
    double s = 0.0;
    for (int l = m + 1; l < j; l++) s += Tab::a(j, l) * Tab::a(l, m);
    return s;
  }
  __host__ __device__ static constexpr double ba(int m) {  // (b A)_m
    double s = 0.0;
    for (int j = m + 1; j < Tab::S; j++) s += Tab::b(j) * Tab::a(j, m);
    return s;
  }
  __host__ __device__ static constexpr double bta(int m) {  // (bt A)_m
    double s = 0.0;
    for (int j = m + 1; j < Tab::S; j++) s += Tab::bt(j) * Tab::a(j, m);
    return s;
  }
};

}  // namespace gs
