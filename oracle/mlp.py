"""FP64 CPU oracle of the learned-start network -- TEST INFRASTRUCTURE ONLY.

The network of the learned initial guess (no counterpart in the paper): features
f (16) standardised as (f - mean) / std, three hidden layers of 64 with SiLU
(s / (1 + e^-s)), a linear output of 3, trained on the mean over rows and outputs
of (out - (label - label_mean) / label_std)^2.  Written plainly in numpy float64
from that definition, with the backward pass derived by hand (chain rule); the
tests pin the backward pass against central finite differences.

Parameter vector order: W1 [64][16], b1 [64], W2 [64][64], b2, W3 [64][64], b3,
W4 [3][64], b4 [3].  Blob layout (32-bit words): header 8, feature mean 16, std
16, label mean 4, std 4, b1 64, b2 64, b3 64, b4 4, then BF16 W1, W2, W3, W4
(4 rows, the last zero).
"""
import numpy as np

NI, NH, NO = 16, 64, 3
SHAPES = [("W1", (NH, NI)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH, NH)), ("b3", (NH,)),
          ("W4", (NO, NH)), ("b4", (NO,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)
MAGIC, VERSION = 0x57534D53, 1
BLOB_WORDS = 244 + (NH * NI + NH * NH * 2 + 4 * NH) // 2


def _bf16_to_f64(u16):
    return (np.asarray(u16, np.uint32) << 16).view(np.float32).astype(np.float64)


def _f32_to_bf16_bits(x):
    """Round-to-nearest-even FP32 -> BF16 bit patterns."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def parse_blob(blob):
    w = np.frombuffer(bytes(blob), dtype=np.uint32)
    assert w.size >= BLOB_WORDS and w[0] == MAGIC and w[1] == VERSION
    f = w.view(np.float32).astype(np.float64)
    p = {"fm": f[8:24], "fs": f[24:40], "ym": f[40:43], "ys": f[44:47],
         "b1": f[48:112], "b2": f[112:176], "b3": f[176:240], "b4": f[240:243]}
    h = np.frombuffer(bytes(blob), dtype=np.uint16)[244 * 2:]
    o = 0
    for name, n in (("W1", NH * NI), ("W2", NH * NH), ("W3", NH * NH), ("W4", 4 * NH)):
        p[name] = _bf16_to_f64(h[o:o + n])
        o += n
    p["W1"] = p["W1"].reshape(NH, NI)
    p["W2"] = p["W2"].reshape(NH, NH)
    p["W3"] = p["W3"].reshape(NH, NH)
    p["W4"] = p["W4"].reshape(4, NH)[:NO]
    return p


def make_blob(params, fm, fs, ym, ys):
    """Blob from a parameter dict (weights are rounded to BF16) and statistics."""
    w = np.zeros(BLOB_WORDS, np.uint32)
    w[0], w[1], w[2], w[3], w[4] = MAGIC, VERSION, NI, NH, NO
    f = w.view(np.float32)
    f[8:24], f[24:40] = fm, fs
    f[40:43], f[43] = ym, 0.0
    f[44:47], f[47] = ys, 1.0
    f[48:112], f[112:176], f[176:240] = params["b1"], params["b2"], params["b3"]
    f[240:243] = params["b4"]
    h = w.view(np.uint16)
    o = 244 * 2
    for name in ("W1", "W2", "W3"):
        bits = _f32_to_bf16_bits(np.asarray(params[name]).ravel())
        h[o:o + bits.size] = bits
        o += bits.size
    h[o:o + NO * NH] = _f32_to_bf16_bits(np.asarray(params["W4"]).ravel())
    return w.tobytes()


def flatten(p):
    return np.concatenate([np.asarray(p[n], np.float64).ravel() for n, _ in SHAPES])


def unflatten(v):
    out, o = {}, 0
    for n, s in SHAPES:
        k = int(np.prod(s))
        out[n] = np.asarray(v[o:o + k], np.float64).reshape(s)
        o += k
    return out


def silu(s):
    return s / (1.0 + np.exp(-s))


def dsilu(s):
    g = 1.0 / (1.0 + np.exp(-s))
    return g * (1.0 + s * (1.0 - g))


def forward(p, feat):
    """Unstandardised outputs for raw feature rows (n, 16)."""
    x = (np.asarray(feat, np.float64) - p["fm"]) / p["fs"]
    a1 = silu(x @ p["W1"].T + p["b1"])
    a2 = silu(a1 @ p["W2"].T + p["b2"])
    a3 = silu(a2 @ p["W3"].T + p["b3"])
    out = a3 @ p["W4"].T + p["b4"]
    return out * p["ys"] + p["ym"]


def loss_and_grad(p, feat, label):
    """Mean over rows and outputs of the squared error of the standardised output,
    and its gradient w.r.t. the parameter vector (order of SHAPES)."""
    x = (np.asarray(feat, np.float64) - p["fm"]) / p["fs"]
    t = (np.asarray(label, np.float64) - p["ym"]) / p["ys"]
    n = x.shape[0]
    z1 = x @ p["W1"].T + p["b1"]
    a1 = silu(z1)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = silu(z2)
    z3 = a2 @ p["W3"].T + p["b3"]
    a3 = silu(z3)
    out = a3 @ p["W4"].T + p["b4"]
    e = out - t
    loss = float(np.mean(e * e))
    g_out = 2.0 * e / (n * NO)                 # d loss / d out
    g = {"W4": g_out.T @ a3, "b4": g_out.sum(0)}
    d3 = (g_out @ p["W4"]) * dsilu(z3)
    g["W3"], g["b3"] = d3.T @ a2, d3.sum(0)
    d2 = (d3 @ p["W3"]) * dsilu(z2)
    g["W2"], g["b2"] = d2.T @ a1, d2.sum(0)
    d1 = (d2 @ p["W2"]) * dsilu(z1)
    g["W1"], g["b1"] = d1.T @ x, d1.sum(0)
    return loss, flatten(g)


def loss_only(p, feat, label):
    x = (np.asarray(feat, np.float64) - p["fm"]) / p["fs"]
    t = (np.asarray(label, np.float64) - p["ym"]) / p["ys"]
    a = silu(x @ p["W1"].T + p["b1"])
    a = silu(a @ p["W2"].T + p["b2"])
    a = silu(a @ p["W3"].T + p["b3"])
    e = a @ p["W4"].T + p["b4"] - t
    return float(np.mean(e * e))


def random_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = {}
    for n, s in SHAPES:
        fan = s[1] if len(s) == 2 else 1
        p[n] = rng.standard_normal(s) * scale / np.sqrt(fan) if len(s) == 2 else 0.1 * rng.standard_normal(s)
    return p
