// Host build of the CUDA path's per-pair math (nep_math.cuh) for CPU tests.
#include "../../paper_2305_08140_gb300/csrc/nep_math.cuh"

extern "C" {

void h_harmonics(double x, double y, double z, double* Y) { nepm::harmonics<double>(x, y, z, Y); }

void h_harmonics_grad_dot(double x, double y, double z, const double* G, double* v)
{
    nepm::harmonics_grad_dot<double>(x, y, z, G, v[0], v[1], v[2]);
}

double h_fourbody(const double* A2, double* dq) { return nepm::fourbody<double>(A2, dq); }

void h_cheb9(double r, double inv_rc, double* T, double* dT, double* out3)
{
    double fc, dfc, dxdr;
    nepm::cheb<9, true, double>(r, inv_rc, T, dT, fc, dfc, dxdr);
    out3[0] = fc; out3[1] = dfc; out3[2] = dxdr;
}

void h_harmonics_f(float x, float y, float z, float* Y) { nepm::harmonics<float>(x, y, z, Y); }
}

extern "C" void h_cutoff_f(float x, float* sc)
{
    nepm::cutoff_sincospi(x, &sc[0], &sc[1]);
}

extern "C" void h_harmonics_dir(const double* u, const double* w, double* D)
{
    nepm::harmonics_dir<double>(u[0], u[1], u[2], w[0], w[1], w[2], D);
}

extern "C" void h_fourbody_hvp(const double* A2, const double* Ad, double* out)
{
    double T[6], Td[6], S[6];
    nepm::fourbody_T<double>(A2, T);
    nepm::fourbody_T<double>(Ad, Td);
    nepm::sym_anticomm<double>(T, Td, S);
    nepm::fourbody_map<double>(S, out);
}

// grouped harmonics and gradient contraction, summed over the three groups
extern "C" void h_harmonics_groups(const double* u, const double* G, double* Y, double* v)
{
    nepm::harmonics_group<0, double>(u[0], u[1], u[2], Y);
    nepm::harmonics_group<1, double>(u[0], u[1], u[2], Y + 8);
    nepm::harmonics_group<2, double>(u[0], u[1], u[2], Y + 16);
    v[0] = v[1] = v[2] = 0.0;
    nepm::harmonics_grad_dot_group<0, double>(u[0], u[1], u[2], G, v[0], v[1], v[2]);
    nepm::harmonics_grad_dot_group<1, double>(u[0], u[1], u[2], G + 8, v[0], v[1], v[2]);
    nepm::harmonics_grad_dot_group<2, double>(u[0], u[1], u[2], G + 16, v[0], v[1], v[2]);
}
