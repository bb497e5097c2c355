"""Force a hierarchy's launch choices through the autotuner's cache file:
tune once into a fresh file, rewrite the chosen values of some levels, and
load the file back (nmg_autotune reads a matching entry instead of timing)."""


def force_tuning(G, batch, path, levels):
    """levels: {level: dict(res=..., rst=..., ref=..., filt=...)} (missing
    keys keep the tuned value)."""
    path = str(path)
    open(path, "w").close()
    G.autotune(batch, path)
    line = open(path).read().strip().splitlines()[-1]
    key, vals = line.split(" | ")
    ents = [v for v in vals.split(";") if v]
    for l, ch in levels.items():
        a, b, c, e = (int(t) for t in ents[l].split(","))
        a, b, c, e = ch.get("res", a), ch.get("rst", b), ch.get("ref", c), ch.get("filt", e)
        ents[l] = f"{a},{b},{c},{e}"
    with open(path, "w") as fp:
        fp.write(key + " | " + "".join(v + ";" for v in ents) + "\n")
    G.autotune(batch, path)
