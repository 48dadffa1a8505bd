"""Algorithmic work per unit of the FP64 path (used for roofline fractions).

Counts are floating-point operations of the discretisation itself, as the kernels evaluate it:
add, sub, mul, div, sqrt, min/max and pow count one each; a fused multiply-add counts two.  They
are not instruction counts (a division or square root expands into several FP64 instructions).

Per face (one axis, one face, 3-D viscous WENO5-Z + HLLC):
  WENO5-Z reconstruction    73 per variable and side (JS: 69); 10 per face
  HLLC (one star branch)   115
  dissipative flux          90 (power-law mu; Sutherland 94; 1-D / 2-D fewer tangential terms)
  TENO6-A reconstruction   165 per variable and side, plus the TENO-A scale sensor and cut-off
                           (27 per variable, shared by both sides); 10 and 5 per face
  sixth-order dissipative  the same terms with six-point interpolations (11) and derivatives (12)
Per cell and axis: one face + the flux difference (3 per variable) = face + 15.
Per cell and stage: primitives 15, centre gradients 6 per component, stage combination about 20.
Per cell and RK3 step: 3 stages + the CFL reduction (about 28).
"""

WENO = {"z": 73, "js": 69}
TENO = 165
TENO_SENSOR = 27
HLLC = 115
PRIM = 15
STAGE = 20
DT = 28


def visc_face(ndim, visc, order=4):
    if visc == "none":
        return 0
    tang = ndim - 1                       # tangential axes with derivative terms
    mu = {"constant": 0, "power": 3, "sutherland": 7}[visc]
    if order == 6:
        return 4 * 11 + 4 * 12 + 22 * tang + 2 + mu + 1 + 9 + 7 + 4
    return 20 + 24 + 10 * tang + 2 + mu + 1 + 9 + 7 + 4


def recon_flops(weno):
    """Reconstruction work of one face (five primitives, both sides)."""
    if weno == "teno6a":
        return 10 * TENO + 5 * TENO_SENSOR
    return 10 * WENO[weno]


def face_flops(ndim, weno, visc, order=4):
    return recon_flops(weno) + HLLC + visc_face(ndim, visc, order)


def cell_axis_flops(ndim, weno, visc, order=4):
    """One face flux plus the flux difference of one cell along one axis (a face-kernel unit)."""
    return face_flops(ndim, weno, visc, order) + 15


def cell_stage_flops(ndim, weno, visc, order=4):
    grad = (8 if order == 6 else 6) * 3 * ndim if visc != "none" else 0
    return ndim * cell_axis_flops(ndim, weno, visc, order) + PRIM + grad + STAGE


def cell_update_flops(ndim, weno, visc, order=4):
    """Algorithmic FP64 flops of one cell over one TVD-RK3 step."""
    return 3 * cell_stage_flops(ndim, weno, visc, order) + DT


def cell_update_bytes(nvar=5, word=8):
    """Compulsory HBM bytes of one cell over one RK3 step with a fully fused stage: stage 1 reads
    Un and writes U1 (2 arrays), stages 2 and 3 read two arrays and write one (3 each)."""
    return 8 * nvar * word


# ---- mixed FP32-flux / FP64-state face kernel (FLUID_PREC_MIXED) ------------------------------
# FP64 per cell and axis: the cell-centre Euler flux from the primitives and the stored
# H = E + p (rho u_n 1, adding the increment to the mass flux 1, three momentum FMAs 6, the
# pressure 1, the energy FMA 2) and the flux difference with its scaling and accumulation (15).
# The cell differences come from the exact FP32 split of the primitives and cost no FP64 work.
# FP32: the WENO5 reconstructions, the HLLC increment in jump form (about 150) and the
# dissipative flux (90).
def mixed_cell_axis_flops64():
    return 1 + 1 + 6 + 1 + 2 + 15


def mixed_cell_axis_flops32(weno="z", visc="power"):
    return 10 * WENO[weno] + 150 + (90 if visc != "none" else 0)


def mixed_face_bytes():
    """Compulsory bytes of one face-kernel launch per cell: FP64 primitives and H 6 x 8 read, the
    FP32 (hi, lo) split of 6 primitives 12 x 4 read, FP32 tangential gradients 4 x 4 read, R read
    and written 2 x 40."""
    return 48 + 48 + 16 + 80
