"""FP64 CPU oracle for the fast spectral Boltzmann collision operator (arXiv:1809.10186).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
leg may import or run anything in this package. The CUDA product path never does.
"""
from .collision import (OraclePlan, b_vhs, default_R, fast_Q, fast_Q_batch, direct_Q,
                        gain_Q, loss_Q, gain_radial_products, G_exact, G_quadrature,
                        F_closed, jvp, vjp, dQ_dgamma, dgamma_plan, bkw_f, bkw_Q, bkw_K,
                        grid_c2, moments, conserved_moments, ssp_rk2, ssp_rk3, entropy)
from .quadrature import gauss_legendre, sphere_rule, antipodal_pairs, sphere_monomial_integral
