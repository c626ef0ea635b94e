// Odometry chaining: the paper's odometry experiment combines consecutive
// scan-to-scan estimates as T_E = T^1_0 T^2_1 ... T^l_(l-1) of their mean
// transforms and combines their covariances with a fourth-order
// approximation.  A pose distribution here is a mean pose T_bar and the
// covariance of the left perturbation xi = [rho; phi] in T = exp(xi^) T_bar.
//
// sicp_pose_distribution turns a particle set into one: the mean pose is the
// point where the particles' perturbations average to zero (fixed-point
// iteration from the pose of their mean parameters, angles by circular
// mean), the covariance the sample covariance of those perturbations.
// sicp_compound combines two independent distributions: mean T1 T2,
// covariance S1 + S2' with S2' = Ad(T1) S2 Ad(T1)^T to second order, plus
// (1/12)(<<S1>> S2' + S2' <<S1>>^T + <<S2'>> S1 + S1 <<S2'>>^T) + B / 4 to
// fourth order, where for 3 x 3 blocks <M> = -tr(M) 1 + M, <<S>> =
// [<S_pp>, <S_rp + S_rp^T>; 0, <S_pp>], and B collects the products
// <A><B> + <B A> of the blocks (rr: translation, pp: rotation, rp: cross).
// Host code in float64.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "../../include/steinicp.h"

namespace {

using M3 = double[3][3];

void hat(const double v[3], M3 H) {
    H[0][0] = 0.0;   H[0][1] = -v[2]; H[0][2] = v[1];
    H[1][0] = v[2];  H[1][1] = 0.0;   H[1][2] = -v[0];
    H[2][0] = -v[1]; H[2][1] = v[0];  H[2][2] = 0.0;
}

void mul3(const M3 A, const M3 B, M3 C) {
    M3 T;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[i][j] = A[i][0] * B[0][j] + A[i][1] * B[1][j] + A[i][2] * B[2][j];
    memcpy(C, T, sizeof T);
}

// C = exp(phi^) and V (the left Jacobian) by Rodrigues' formula; series below 1e-6 rad.
void so3_exp(const double phi[3], M3 C, M3 V) {
    const double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2], th = sqrt(th2);
    double a, b, c;
    if (th < 1e-6) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
        c = 1.0 / 6.0 - th2 / 120.0;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
        c = (th - sin(th)) / (th2 * th);
    }
    M3 K, K2;
    hat(phi, K);
    mul3(K, K, K2);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double I = i == j ? 1.0 : 0.0;
            C[i][j] = I + a * K[i][j] + b * K2[i][j];
            V[i][j] = I + b * K[i][j] + c * K2[i][j];
        }
}

// phi with exp(phi^) = C, |phi| in [0, pi].
void so3_log(const M3 C, double phi[3]) {
    const double cs = fmin(1.0, fmax(-1.0, (C[0][0] + C[1][1] + C[2][2] - 1.0) / 2.0));
    const double th = acos(cs);
    const double w[3] = {C[2][1] - C[1][2], C[0][2] - C[2][0], C[1][0] - C[0][1]};
    if (th < 1e-6) {
        for (int a = 0; a < 3; ++a) phi[a] = 0.5 * (1.0 + th * th / 6.0) * w[a];
    } else if (M_PI - th < 1e-6) {
        // near pi: the axis is the dominant column of (C + 1) / 2 = a a^T
        int k = 0;
        for (int a = 1; a < 3; ++a)
            if (C[a][a] > C[k][k]) k = a;
        double ax[3] = {C[0][k], C[1][k], C[2][k]};
        ax[k] += 1.0;
        const double n = sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
        double sgn = ax[0] * w[0] + ax[1] * w[1] + ax[2] * w[2] < 0.0 ? -1.0 : 1.0;
        for (int a = 0; a < 3; ++a) phi[a] = sgn * th * ax[a] / n;
    } else {
        const double s = th / (2.0 * sin(th));
        for (int a = 0; a < 3; ++a) phi[a] = s * w[a];
    }
}

struct Pose {
    M3 C;
    double r[3];
};

void se3_exp(const double xi[6], Pose& T) {
    M3 V;
    so3_exp(xi + 3, T.C, V);
    for (int i = 0; i < 3; ++i) T.r[i] = V[i][0] * xi[0] + V[i][1] * xi[1] + V[i][2] * xi[2];
}

// V^-1 rho = r by Gaussian elimination on the 3 x 3 left Jacobian.
void solve3(const M3 A, const double b[3], double x[3]) {
    double M[3][4];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) M[i][j] = A[i][j];
        M[i][3] = b[i];
    }
    for (int c = 0; c < 3; ++c) {
        int p = c;
        for (int i = c + 1; i < 3; ++i)
            if (fabs(M[i][c]) > fabs(M[p][c])) p = i;
        for (int j = 0; j < 4; ++j) {
            const double t = M[c][j];
            M[c][j] = M[p][j];
            M[p][j] = t;
        }
        for (int i = 0; i < 3; ++i)
            if (i != c) {
                const double f = M[i][c] / M[c][c];
                for (int j = c; j < 4; ++j) M[i][j] -= f * M[c][j];
            }
    }
    for (int i = 0; i < 3; ++i) x[i] = M[i][3] / M[i][i];
}

void se3_log(const Pose& T, double xi[6]) {
    so3_log(T.C, xi + 3);
    M3 C, V;
    so3_exp(xi + 3, C, V);
    solve3(V, T.r, xi);
}

void compose(const Pose& A, const Pose& B, Pose& out) {
    Pose o;
    mul3(A.C, B.C, o.C);
    for (int i = 0; i < 3; ++i) o.r[i] = A.C[i][0] * B.r[0] + A.C[i][1] * B.r[1] + A.C[i][2] * B.r[2] + A.r[i];
    out = o;
}

void inverse(const Pose& A, Pose& out) {
    Pose o;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) o.C[i][j] = A.C[j][i];
    for (int i = 0; i < 3; ++i) o.r[i] = -(o.C[i][0] * A.r[0] + o.C[i][1] * A.r[1] + o.C[i][2] * A.r[2]);
    out = o;
}

// Particle parameters (x, y, z, roll, pitch, yaw) -> pose, C = Rz(yaw) Ry(pitch) Rx(roll).
void pose_of(const double th[6], Pose& T) {
    const double cr = cos(th[3]), sr = sin(th[3]), cp = cos(th[4]), sp = sin(th[4]), cy = cos(th[5]), sy = sin(th[5]);
    const M3 X = {{1, 0, 0}, {0, cr, -sr}, {0, sr, cr}};
    const M3 Y = {{cp, 0, sp}, {0, 1, 0}, {-sp, 0, cp}};
    const M3 Z = {{cy, -sy, 0}, {sy, cy, 0}, {0, 0, 1}};
    M3 ZY;
    mul3(Z, Y, ZY);
    mul3(ZY, X, T.C);
    for (int i = 0; i < 3; ++i) T.r[i] = th[i];
}

void to_mat4(const Pose& T, double* M) {
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) M[4 * i + j] = T.C[i][j];
        M[4 * i + 3] = T.r[i];
    }
    M[12] = M[13] = M[14] = 0.0;
    M[15] = 1.0;
}

bool from_mat4(const double* M, Pose& T) {
    for (int i = 0; i < 16; ++i)
        if (!isfinite(M[i])) return false;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) T.C[i][j] = M[4 * i + j];
        T.r[i] = M[4 * i + 3];
    }
    // a rotation: C C^T = 1 and det C = 1 to 1e-6
    M3 Ct, P;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Ct[i][j] = T.C[j][i];
    mul3(T.C, Ct, P);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (fabs(P[i][j] - (i == j ? 1.0 : 0.0)) > 1e-6) return false;
    const double det = T.C[0][0] * (T.C[1][1] * T.C[2][2] - T.C[1][2] * T.C[2][1]) -
                       T.C[0][1] * (T.C[1][0] * T.C[2][2] - T.C[1][2] * T.C[2][0]) +
                       T.C[0][2] * (T.C[1][0] * T.C[2][1] - T.C[1][1] * T.C[2][0]);
    return fabs(det - 1.0) <= 1e-6 && fabs(M[12]) + fabs(M[13]) + fabs(M[14]) + fabs(M[15] - 1.0) <= 1e-12;
}

using M6 = double[6][6];

// <M> = -tr(M) 1 + M on a 3 x 3 block
void angle3(const M3 M, M3 out) {
    const double t = M[0][0] + M[1][1] + M[2][2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) out[i][j] = M[i][j] - (i == j ? t : 0.0);
}

void block(const M6 S, int r0, int c0, M3 out) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) out[i][j] = S[r0 + i][c0 + j];
}

// <A><B> + <B A>
void bterm(const M3 A, const M3 B, M3 out) {
    M3 a, b, ab, ba, bba;
    angle3(A, a);
    angle3(B, b);
    mul3(a, b, ab);
    mul3(B, A, ba);
    angle3(ba, bba);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) out[i][j] = ab[i][j] + bba[i][j];
}

void transpose3(const M3 A, M3 out) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) out[i][j] = A[j][i];
}

// <<S>> = [<S_pp>, <S_rp + S_rp^T>; 0, <S_pp>]
void angle6(const M6 S, M6 out) {
    M3 pp, rp, rpt, a, b;
    block(S, 3, 3, pp);
    block(S, 0, 3, rp);
    transpose3(rp, rpt);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) rp[i][j] += rpt[i][j];
    angle3(pp, a);
    angle3(rp, b);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) out[i][j] = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            out[i][j] = a[i][j];
            out[i][3 + j] = b[i][j];
            out[3 + i][3 + j] = a[i][j];
        }
}

void mul6(const M6 A, const M6 B, M6 C) {
    M6 T;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double s = 0.0;
            for (int k = 0; k < 6; ++k) s += A[i][k] * B[k][j];
            T[i][j] = s;
        }
    memcpy(C, T, sizeof T);
}

void adjoint(const Pose& T, M6 A) {
    M3 rh, rc;
    hat(T.r, rh);
    mul3(rh, T.C, rc);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) A[i][j] = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            A[i][j] = T.C[i][j];
            A[3 + i][3 + j] = T.C[i][j];
            A[i][3 + j] = rc[i][j];
        }
}

bool finite_n(const double* a, int n) {
    for (int i = 0; i < n; ++i)
        if (!isfinite(a[i])) return false;
    return true;
}

}  // namespace

extern "C" int sicp_pose_distribution(const float* particles, int32_t K, double* T_mean, double* cov) {
    if (!particles || !T_mean || !cov || K < 1 || K > (1 << 20)) return SICP_EINVAL;
    std::vector<Pose> Ts(K);
    double mean_t[3] = {0, 0, 0}, ss[3] = {0, 0, 0}, sc[3] = {0, 0, 0};
    for (int32_t j = 0; j < K; ++j) {
        double th[6];
        for (int a = 0; a < 6; ++a) {
            th[a] = (double)particles[6 * j + a];
            if (!isfinite(th[a])) return SICP_EINVAL;
        }
        pose_of(th, Ts[j]);
        for (int a = 0; a < 3; ++a) {
            mean_t[a] += th[a];
            ss[a] += sin(th[3 + a]);
            sc[a] += cos(th[3 + a]);
        }
    }
    // start: the pose of the mean parameters (angles by circular mean)
    double th0[6];
    for (int a = 0; a < 3; ++a) {
        th0[a] = mean_t[a] / K;
        th0[3 + a] = (ss[a] == 0.0 && sc[a] == 0.0) ? 0.0 : atan2(ss[a], sc[a]);
    }
    Pose Tb, Tbi, D;
    pose_of(th0, Tb);
    std::vector<double> xi(6 * (size_t)K);
    for (int it = 0; it < 100; ++it) {
        inverse(Tb, Tbi);
        double step[6] = {0, 0, 0, 0, 0, 0};
        for (int32_t j = 0; j < K; ++j) {
            compose(Ts[j], Tbi, D);
            se3_log(D, &xi[6 * j]);
            for (int a = 0; a < 6; ++a) step[a] += xi[6 * j + a];
        }
        double mx = 0.0;
        for (int a = 0; a < 6; ++a) {
            step[a] /= K;
            mx = fmax(mx, fabs(step[a]));
        }
        if (mx < 1e-15) break;
        Pose E;
        se3_exp(step, E);
        compose(E, Tb, Tb);
    }
    inverse(Tb, Tbi);
    for (int32_t j = 0; j < K; ++j) {
        compose(Ts[j], Tbi, D);
        se3_log(D, &xi[6 * j]);
    }
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) {
            double s = 0.0;
            for (int32_t j = 0; j < K; ++j) s += xi[6 * j + a] * xi[6 * j + b];
            cov[6 * a + b] = K > 1 ? s / (double)(K - 1) : 0.0;
        }
    to_mat4(Tb, T_mean);
    return SICP_OK;
}

extern "C" int sicp_compound(const double* T1, const double* cov1, const double* T2, const double* cov2,
                             int32_t order, double* T_out, double* cov_out) {
    if (!T1 || !cov1 || !T2 || !cov2 || !T_out || !cov_out || (order != 2 && order != 4)) return SICP_EINVAL;
    if (!finite_n(cov1, 36) || !finite_n(cov2, 36)) return SICP_EINVAL;
    Pose A, B, C;
    if (!from_mat4(T1, A) || !from_mat4(T2, B)) return SICP_EINVAL;
    M6 S1, S2, Ad, AdT, S2p, S;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            S1[i][j] = cov1[6 * i + j];
            S2[i][j] = cov2[6 * i + j];
        }
    adjoint(A, Ad);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) AdT[i][j] = Ad[j][i];
    mul6(Ad, S2, S2p);
    mul6(S2p, AdT, S2p);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) S[i][j] = S1[i][j] + S2p[i][j];
    if (order == 4) {
        M6 a1, a2, t1, t2, t3, t4;
        angle6(S1, a1);
        angle6(S2p, a2);
        mul6(a1, S2p, t1);
        mul6(a2, S1, t3);
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                t2[i][j] = t1[j][i];   // S2' <<S1>>^T = (<<S1>> S2')^T for symmetric S2'
                t4[i][j] = t3[j][i];
            }
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) S[i][j] += (t1[i][j] + t2[i][j] + t3[i][j] + t4[i][j]) / 12.0;
        M3 s1rr, s1rp, s1pp, s2rr, s2rp, s2pp, s1pr, s2pr, x, y, z, w;
        block(S1, 0, 0, s1rr);
        block(S1, 0, 3, s1rp);
        block(S1, 3, 3, s1pp);
        block(S2p, 0, 0, s2rr);
        block(S2p, 0, 3, s2rp);
        block(S2p, 3, 3, s2pp);
        transpose3(s1rp, s1pr);
        transpose3(s2rp, s2pr);
        M3 Brr, Brp, Bpp;
        bterm(s1pp, s2rr, x);
        bterm(s1pr, s2rp, y);
        bterm(s1rp, s2pr, z);
        bterm(s1rr, s2pp, w);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Brr[i][j] = x[i][j] + y[i][j] + z[i][j] + w[i][j];
        bterm(s1pp, s2pr, x);
        bterm(s1pr, s2pp, y);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Brp[i][j] = x[i][j] + y[i][j];
        bterm(s1pp, s2pp, Bpp);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                S[i][j] += Brr[i][j] / 4.0;
                S[i][3 + j] += Brp[i][j] / 4.0;
                S[3 + i][j] += Brp[j][i] / 4.0;
                S[3 + i][3 + j] += Bpp[i][j] / 4.0;
            }
    }
    compose(A, B, C);
    to_mat4(C, T_out);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) cov_out[6 * i + j] = S[i][j];
    return SICP_OK;
}
