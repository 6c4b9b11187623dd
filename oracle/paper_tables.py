"""The coefficient tables the paper prints, typed in from the paper.

TEST INFRASTRUCTURE ONLY (oracle side).  The product library keeps its own
copy of the two rationals; the two copies are never shared.

Coefficients are in increasing powers of the argument (a_0 .. a_p), as printed.
"""

# Table 1 (tab_arcsin_arccos), Sec. 3.1: fourth degree minimax polynomials.
# ARCSIN row: the function 2*arcsin(tau/sqrt(2)) of tau = sqrt(1 - z) on
#   [0, 1/sqrt(2)] (the substitution that saves two multiplications);
# ARCCOS row: arccos(z); the interval is not printed, [0, 0.5] reproduces it
#   (the identity above is used for z >= 0.5).
TABLE1_ARCSIN_EPS = 2.097814e-05
TABLE1_ARCSIN = [2.097797e-05, 1.412840, 1.429881e-02, 6.704361e-02, 6.909677e-02]
TABLE1_ARCCOS_EPS = 1.048949e-05
TABLE1_ARCCOS = [1.570786, -9.990285e-01, -1.429899e-02, -9.481335e-02, -1.381942e-01]

# Table 2 (tab_exp_poly), Sec. 3.2: minimax polynomials of exp(-z) on [0, 10].
TABLE2_EXP = {
    2: (1.785517e-01, [8.214528e-01, -3.186948e-01, 2.544088e-02]),
    3: (8.259345e-02, [9.174126e-01, -5.631179e-01, 1.015041e-01, -5.519183e-03]),
    4: (3.337085e-02, [9.666313e-01, -7.620584e-01, 2.145386e-01, -2.509526e-02,
                       1.032877e-03]),
}

# Table tab_exp_rat, Sec. 3.2: (4,4) minimax rational of exp(-z) on [0, 10].
EXP_RATIONAL_EPS = 2.227050e-06
EXP_RATIONAL_NUM = [3.206619e-02, -1.195191e-02, 1.756974e-03, -1.199261e-04, 3.182685e-06]
EXP_RATIONAL_DEN = [3.206627e-02, 2.011147e-02, 5.853684e-03, 9.780143e-04, 1.251598e-04]

# Table tab_ent_rat, Sec. 3.3: (4,4) minimax rational of z log z on [0.05, 1].
ENT_RATIONAL_EPS = 7.342477e-07
ENT_RATIONAL_NUM = [-1.519742e-04, -6.835769e-02, -8.856923e-01, -5.369609e-01, 1.491165]
ENT_RATIONAL_DEN = [1.532270e-02, 3.987796e-01, 1.461793, 6.827004e-01, -4.469776e-02]

# Cut-offs and constants stated in Sec. 3.2 - 3.3.
EXP_CUTOFF = 10.0        # Sec. 3.2: exp(-z) returns 0 outside [0, T], T = 10
EXP_AT_CUTOFF = 4.539993e-05  # printed value of e^-T
ENT_CUTOFF = 0.05        # Sec. 3.3: z log z returns 0 below T = 0.05
KAPPA = 0.33             # Sec. 3.2: kernel-width scaling factor
