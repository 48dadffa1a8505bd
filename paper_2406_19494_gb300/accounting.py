"""Algorithmic work per unit of the FP64 path (used for roofline fractions).

The algorithmic counts are measured, not estimated: the oracle's own right-hand side, RK3
combination and CFL rates run on counting scalars (the graph of operations reachable from the
results, so the unselected HLLC branches and discarded halo work do not count; add, sub, mul, div,
sqrt and pow count one each), stored per workload and phase in profiles/oracle_op_counts.json.
`measured_counts()` reads them; the functions below take the measured figure wherever it exists
(3-D WENO5-JS / WENO5-Z with power-law or Sutherland viscosity or none, and TENO6-A with sixth-order
dissipative fluxes) and fall back to the hand count of this module's table otherwise.

The executed work of the kernels (FP64 instructions counted by ncu on the 64^3 Taylor-Green and
96 x 64 x 64 channel workloads: flops = 2 DFMA + DADD + DMUL) is kept beside it in EXECUTED.  The
kernels share WENO5 indicator sets between neighbouring faces, so they execute fewer flops than
the definition needs; TENO6-A's definition as the oracle writes it evaluates its smoothness
measures as full quadratic forms (each symmetric pair twice), which no implementation does, so for
that kernel the executed count is the meaningful one.

Hand counts (the fallback):

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

import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COUNTS = os.path.join(ROOT, "profiles", "oracle_op_counts.json")

# executed FP64 flops per cell and axis (ncu op counters, 2 DFMA + DADD + DMUL) of the face kernels
EXECUTED = {"k_face": 741, "k_face_teno": 1561}

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


_measured = None


def measured_counts():
    """The oracle's counted work per workload (None if the file is missing)."""
    global _measured
    if _measured is None:
        try:
            with open(COUNTS) as f:
                _measured = json.load(f)["workloads"]
        except (OSError, ValueError, KeyError):
            _measured = {}
    return _measured


def _key(ndim, weno, visc, order):
    if ndim != 3:
        return None
    if weno == "teno6a":
        return "teno6a_power_visc6" if (visc == "power" and order == 6) else None
    base = {"z": "weno5z", "js": "weno5js"}.get(weno)
    if base is None or order != 4:
        return None
    return {"power": base + "_power", "none": "weno5z_euler" if weno == "z" else None,
            "sutherland": "weno5z_sutherland" if weno == "z" else None}.get(visc)


def measured(ndim, weno, visc, unit, order=4):
    """Counted flops of `unit` (cell_axis, cell_update, face, ...) or None."""
    k = _key(ndim, weno, visc, order)
    m = measured_counts().get(k) if k else None
    return m[unit]["flops"] if m else None


def cell_axis_flops(ndim, weno, visc, order=4):
    """One face flux plus the flux difference of one cell along one axis (a face-kernel unit)."""
    m = measured(ndim, weno, visc, "cell_axis", order)
    return m if m is not None else face_flops(ndim, weno, visc, order) + 15


def cell_stage_flops(ndim, weno, visc, order=4):
    grad = (8 if order == 6 else 6) * 3 * ndim if visc != "none" else 0
    return ndim * cell_axis_flops(ndim, weno, visc, order) + PRIM + grad + STAGE


def cell_update_flops(ndim, weno, visc, order=4):
    """Algorithmic FP64 flops of one cell over one TVD-RK3 step."""
    m = measured(ndim, weno, visc, "cell_update", order)
    return m if m is not None else 3 * cell_stage_flops(ndim, weno, visc, order) + DT


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
