"""IMEX ARK (ESDIRK) Butcher tableaux used by the oracle (Sec. 6).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Each tableau is (A explicit, At implicit, b = bt), Sec. 4.1: A strictly lower
triangular, At lower triangular with a zero first row (explicit first stage)
and a constant diagonal gamma.  The paper names the methods but prints no
coefficients, so they are taken from the cited constructions and pinned by
their order conditions and observed convergence order in the tests:

  ARK2  ARK(2,3,2)b of Giraldo, Kelly & Constantinescu (2013) with a32 = 1/2,
        gamma = 1 - 1/sqrt(2).
  ARK3  ARK3(2)4L[2]SA of Kennedy & Carpenter (2003).
  ARK4  ARK4(3)6L[2]SA of Kennedy & Carpenter (2003).
  ARS3  ARK(3,4,3) of Ascher, Ruuth & Spiteri (1997) (Sec. 6 names it ARS3):
        gamma the root in (1/6, 1/2) of 6 g^3 - 18 g^2 + 9 g - 1 = 0, the
        construction's free explicit coefficients a42 = a43 = 0.5529291480359398,
        a31 and a32 from its closed forms in gamma, a42 and a43; the implicit
        part has a zero first column.
"""

from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction as Fr
import math

import numpy as np


@dataclass(frozen=True)
class Tableau:
    name: str
    order: int
    A: np.ndarray   # explicit, s x s
    At: np.ndarray  # implicit, s x s
    b: np.ndarray   # weights, shared by both parts

    @property
    def s(self) -> int:
        return len(self.b)

    @property
    def gamma(self) -> float:
        return float(self.At[1, 1])

    @property
    def c(self) -> np.ndarray:
        return self.A.sum(axis=1)


def _ark2() -> Tableau:
    g = 1.0 - 1.0 / math.sqrt(2.0)
    d = 1.0 / (2.0 * math.sqrt(2.0))
    A = np.array([[0, 0, 0], [2 * g, 0, 0], [0.5, 0.5, 0]], dtype=np.float64)
    At = np.array([[0, 0, 0], [g, g, 0], [d, d, g]], dtype=np.float64)
    b = np.array([d, d, g])
    return Tableau("ARK2", 2, A, At, b)


def _to_np(M) -> np.ndarray:
    return np.array([[float(x) for x in row] for row in M], dtype=np.float64)


def _ark3() -> Tableau:
    g = Fr(1767732205903, 4055673282236)
    b = [Fr(1471266399579, 7840856788654), Fr(-4482444167858, 7529755066697),
         Fr(11266239266428, 11593286722821), g]
    At = [[Fr(0)] * 4 for _ in range(4)]
    At[1][:2] = [g, g]
    At[2][:3] = [Fr(2746238789719, 10658868560708), Fr(-640167445237, 6845629431997), g]
    At[3] = list(b)
    A = [[Fr(0)] * 4 for _ in range(4)]
    A[1][0] = Fr(1767732205903, 2027836641118)
    A[2][:2] = [Fr(5535828885825, 10492691773637), Fr(788022342437, 10882634858940)]
    A[3][:3] = [Fr(6485989280629, 16251701735622), Fr(-4246266847089, 9704473918619),
                Fr(10755448449292, 10357097424841)]
    return Tableau("ARK3", 3, _to_np(A), _to_np(At), np.array([float(x) for x in b]))


def _ark4() -> Tableau:
    g = Fr(1, 4)
    b = [Fr(82889, 524892), Fr(0), Fr(15625, 83664), Fr(69875, 102672), Fr(-2260, 8211), g]
    At = [[Fr(0)] * 6 for _ in range(6)]
    At[1][:2] = [g, g]
    At[2][:3] = [Fr(8611, 62500), Fr(-1743, 31250), g]
    At[3][:4] = [Fr(5012029, 34652500), Fr(-654441, 2922500), Fr(174375, 388108), g]
    At[4][:5] = [Fr(15267082809, 155376265600), Fr(-71443401, 120774400),
                 Fr(730878875, 902184768), Fr(2285395, 8070912), g]
    At[5] = list(b)
    A = [[Fr(0)] * 6 for _ in range(6)]
    A[1][0] = Fr(1, 2)
    A[2][:2] = [Fr(13861, 62500), Fr(6889, 62500)]
    A[3][:3] = [Fr(-116923316275, 2393684061468), Fr(-2731218467317, 15368042101831),
                Fr(9408046702089, 11113171139209)]
    A[4][:4] = [Fr(-451086348788, 2902428689909), Fr(-2682348792572, 7519795681897),
                Fr(12662868775082, 11960479115383), Fr(3355817975965, 11060851509271)]
    A[5][:5] = [Fr(647845179188, 3216320057751), Fr(73281519250, 8382639484533),
                Fr(552539513391, 3454668386233), Fr(3354512671639, 8306763924573),
                Fr(4040, 17871)]
    return Tableau("ARK4", 4, _to_np(A), _to_np(At), np.array([float(x) for x in b]))


def _ars3() -> Tableau:
    g = 0.4358665215  # Newton on the cubic from the published 10-digit value
    for _ in range(4):
        g -= (6 * g ** 3 - 18 * g ** 2 + 9 * g - 1) / (18 * g ** 2 - 36 * g + 9)
    a42 = a43 = 0.5529291480359398
    b1 = -1.5 * g * g + 4.0 * g - 0.25
    b2 = 1.5 * g * g - 5.0 * g + 1.25
    a31 = ((1 - 4.5 * g + 1.5 * g * g) * a42 + (2.75 - 10.5 * g + 3.75 * g * g) * a43
           - 3.5 + 13 * g - 4.5 * g * g)
    a32 = ((-1 + 4.5 * g - 1.5 * g * g) * a42 + (-2.75 + 10.5 * g - 3.75 * g * g) * a43
           + 4 - 12.5 * g + 4.5 * g * g)
    A = np.array([[0, 0, 0, 0], [g, 0, 0, 0], [a31, a32, 0, 0], [1 - a42 - a43, a42, a43, 0]])
    At = np.array([[0, 0, 0, 0], [0, g, 0, 0], [0, (1 - g) / 2, g, 0], [0, b1, b2, g]])
    return Tableau("ARS3", 3, A, At, np.array([0.0, b1, b2, g]))


ARK2 = _ark2()
ARK3 = _ark3()
ARK4 = _ark4()
ARS3 = _ars3()
ALL = {t.name: t for t in (ARK2, ARK3, ARK4, ARS3)}
