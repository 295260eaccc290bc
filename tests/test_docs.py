"""Every repository path that README.md cite in backticks exists (globs and
brace patterns aside), so the file map and the profile references stay current."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PATH = re.compile(r"`((?:profiles|tests|oracle|include|paper_1309_6250_gb300|csrc)/[^`\s]+)`")


def test_cited_paths_exist():
    missing = []
    for doc in ("DESIGN.md", "README.md"):
        with open(os.path.join(ROOT, doc)) as f:
            text = f.read()
        for ref in sorted(set(PATH.findall(text))):
            path = ref.split(":")[0]
            if any(c in path for c in "*{"):
                continue
            if not any(os.path.exists(os.path.join(ROOT, base, path)) for base in ("", "paper_1309_6250_gb300")):
                missing.append((doc, ref))
    assert not missing, missing
