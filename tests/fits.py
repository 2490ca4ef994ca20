"""Rate estimators for mode histories (test helpers; no PIC arithmetic).

``pencil`` is the matrix-pencil method (Hua and Sarkar, 1990): it writes a
uniformly sampled complex signal as a sum of M complex exponentials
a_i exp(s_i t) and returns the exponents s_i and amplitudes a_i, so a growing
or damped root can be separated from the other roots present in the same
Fourier mode.  ``damped_cosine`` is the classic least-squares fit of
A exp(g t) cos(w t + phi) to the real part of a mode signal.
"""
import numpy as np


def pencil(c, dt, M=3):
    """Exponents s (complex, per unit time) and amplitudes of c_n ~ sum a_i exp(s_i n dt)."""
    c = np.asarray(c, dtype=np.complex128)
    N = len(c)
    L = N // 2
    Y = np.array([c[i:i + L + 1] for i in range(N - L)])
    _, _, Vh = np.linalg.svd(Y, full_matrices=False)
    V = Vh[:M].conj().T
    z = np.linalg.eigvals(np.linalg.pinv(V[:-1]) @ V[1:])
    s = np.log(z) / dt
    Z = np.vander(z, N, increasing=True).T
    a = np.linalg.lstsq(Z, c, rcond=None)[0]
    return s, a


def fastest_root(t, c, t0, t1, M=3):
    """(growth rate, |frequency|) of the most strongly growing pencil root on [t0, t1]."""
    t = np.asarray(t)
    sel = (t >= t0) & (t <= t1)
    s, _ = pencil(np.asarray(c)[sel], t[1] - t[0], M)
    i = int(np.argmax(s.real))
    return s[i].real, abs(s[i].imag)


def damped_cosine(t, c, t0, t1, guess):
    """(g, |w|) of A exp(g t) cos(w t + phi) fitted to Re(c e^{-i arg c_0}) on (t0, t1)."""
    from scipy.optimize import curve_fit

    t = np.asarray(t)
    c = np.asarray(c)
    sig = (c * np.exp(-1j * np.angle(c[0]))).real
    sel = (t > t0) & (t < t1)

    def model(tt, A, g, om, ph):
        return A * np.exp(g * tt) * np.cos(om * tt + ph)

    popt, _ = curve_fit(model, t[sel], sig[sel],
                        p0=[np.max(np.abs(sig[sel])), guess.imag, guess.real, 0.0], maxfev=20000)
    return popt[1], abs(popt[2])
