"""Writes disc_arc_lengths.json: exact line integrals of a uniform disc over circles.

For a disc of amplitude a, radius rho and centre c, and a circle of radius r around a
detector at distance D_c from c, the part of the circle inside the disc is an arc of
angle 2*theta with cos(theta) = (D_c^2 + r^2 - rho^2) / (2 D_c r), so the integral of
the disc indicator over the circle (eq. (K_def), a line integral) is 2 a r theta.  The
whole circle lies inside when D_c + r <= rho and misses the disc when r + rho <= D_c or
D_c + rho <= r.  Only the standard library is used.
"""
import json
import math
import os

PHANTOM = (0.15, -0.1, 0.45, 0.8)       # cx, cy, rho, amplitude
DETECTORS = [(1.2, 0.0), (0.0, -1.2), (-0.9, 0.7)]
R_FIRST, DR, N_R = 0.3, 0.0875, 25


def arc_integral(det, r, cx, cy, rho, amp):
    dc = math.hypot(det[0] - cx, det[1] - cy)
    if dc + r <= rho:
        return amp * 2 * math.pi * r
    if r + rho <= dc or dc + rho <= r:
        return 0.0
    c = (dc * dc + r * r - rho * rho) / (2 * dc * r)
    return amp * 2 * r * math.acos(max(-1.0, min(1.0, c)))


def main():
    radii = [R_FIRST + k * DR for k in range(N_R)]
    cases = []
    for d, det in enumerate(DETECTORS):
        for r in radii:
            cases.append({"d": d, "det": list(det), "r": r, "disc": list(PHANTOM),
                          "value": arc_integral(det, r, *PHANTOM)})
    out = {"source": "closed-form circle-disc arc length, eq. (K_def) line integral",
           "phantom": list(PHANTOM), "detectors": [list(d) for d in DETECTORS],
           "radii": radii, "cases": cases}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "disc_arc_lengths.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
